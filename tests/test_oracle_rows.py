"""Pins for the oracle's row helpers (Sec. 3.3, eq. matrixelmemts).

``nystrom.dense_rows`` and ``nystrom.dense_row_block`` give the expected values of
the sampled-row checks at sizes where the dense matrix is out of reach (the
65,536-point three-layer workload, the stored rows of the million-point
four-layer workload).  Here they must equal the rows and entries of
``nystrom.dense_matrix`` itself on media with density contrast, where
G_{l l'}(r, r') != G_{l' l}(r', r): a transposed field/source slot, a self term
on the wrong column, a dropped reaction part or a wrong layer wavenumber in
either helper fails these tests.
"""

import numpy as np
import pytest

from oracle import nystrom
from workloads import Medium, circle, ellipse


def _case(n_layers):
    if n_layers == 2:
        med = Medium(interfaces=[0.0], k=[2.0, 3.5], eta=[1.0, 2.5])
        bodies = [circle(0.0, 0.1, 0.45, 40), ellipse(1.3, -0.7, 0.35, 0.2, 0.4, 32)]
    else:
        med = Medium(interfaces=[0.0, -1.2], k=[3.0, 5.0, 2.5], eta=[1.0, 3.0, 1.7])
        bodies = [circle(-0.6, 0.05, 0.4, 36), ellipse(0.8, -1.15, 0.45, 0.3, 0.9, 40),
                  circle(0.2, -2.0, 0.3, 24)]
    pts, w, _, _ = nystrom.elements(bodies)
    return med, pts, w


@pytest.fixture(scope="module", params=[2, 3])
def dense(request):
    med, pts, w = _case(request.param)
    K = nystrom.dense_matrix(med, pts, w)
    lay = nystrom.layer_of(med, pts[:, 1])
    # every layer of the medium holds points, and the rows below reach all of them
    assert np.unique(lay).size == request.param
    return med, pts, w, K, lay


def _rows(lay, rng):
    rows = [int(rng.choice(np.flatnonzero(lay == l))) for l in np.unique(lay)]
    rows += [0, lay.size - 1]
    return np.array(sorted(set(rows)), dtype=np.int64)


def test_dense_rows_equal_the_dense_matrix(dense):
    med, pts, w, K, lay = dense
    rows = _rows(lay, np.random.default_rng(3))
    R = nystrom.dense_rows(med, pts, w, rows)
    scale = np.abs(K).max()
    np.testing.assert_allclose(R, K[rows], rtol=0, atol=1e-14 * scale)
    # the diagonal (self term plus the self-image reaction) sits in the row's own column
    np.testing.assert_allclose(R[np.arange(rows.size), rows], np.diag(K)[rows], rtol=0, atol=1e-14 * scale)


def test_dense_row_block_equals_the_dense_matrix(dense):
    med, pts, w, K, lay = dense
    rng = np.random.default_rng(5)
    scale = np.abs(K).max()
    for r in _rows(lay, rng):
        # a random subset of columns that includes the row's own column and columns of every layer
        cols = np.unique(np.concatenate([rng.choice(lay.size, lay.size // 3, replace=False), [r]]))
        rng.shuffle(cols)
        v = nystrom.dense_row_block(med, pts, w, int(r), cols)
        np.testing.assert_allclose(v, K[r, cols], rtol=0, atol=1e-14 * scale)


def test_density_contrast_makes_the_transposition_visible(dense):
    # the pins above could not see a swapped field/source slot if K were symmetric
    # up to the weights; with eta contrast it is not (eta_l G_{l l'}(r, r') =
    # eta_l' G_{l' l}(r', r), Sec. 3.1)
    med, pts, w, K, lay = dense
    Kg = K / w[None, :]
    asym = np.abs(Kg - Kg.T)
    np.fill_diagonal(asym, 0.0)
    assert asym.max() > 1e-3 * np.abs(Kg).max()
