// devmath_harness.cpp -- evaluates the library's own device math (csrc/devmath.cuh,
// compiled here for the host) so that CPU tests can compare it with the oracle and
// with scipy: the interface-referenced reaction densities Sigma_c(lambda) and the
// Bessel/Hankel sequences used by the expansions.
//
//   devmath_harness sigma  <input> <output>
//     input : int32 nl; float64 yint[nl-1], k[nl], eta[nl]; int32 nq;
//             nq x (int32 field layer, arrival, source layer, departure; float64 re, im)
//     output: nq x complex128 Sigma values
//   devmath_harness bessel <input> <output>
//     input : int32 nx, p; float64 x[nx]
//     output: nx x (p+1) float64 J_n(x), then nx x (p+1) complex128 H_n^(1)(x)
//   devmath_harness free <input> <output>
//     input : int32 nq; nq x float64 (k, dx, dy, cf, nx, ny)   (cf: 0 or 1)
//     output: nq x complex128 free-space Nystrom kernel values
//   devmath_harness self <input> <output>
//     input : int32 nq; nq x float64 (k, w, cf)
//     output: nq x complex128 diagonal entries
#include <cstdio>
#include <cstring>
#include <vector>

#include "devmath.cuh"

template <class T>
static bool rd(FILE* f, T* v, size_t n) {
    return std::fread(v, sizeof(T), n, f) == n;
}

static int run_sigma(FILE* in, FILE* out) {
    int32_t nl = 0;
    if (!rd(in, &nl, 1) || nl < 1 || nl > LFMM_MAXLAY) return 2;
    MediumDev m{};
    m.nl = nl;
    if (!rd(in, m.yint, (size_t)(nl - 1)) || !rd(in, m.k, (size_t)nl) || !rd(in, m.eta, (size_t)nl)) return 2;
    m.kmax = 0.0;
    for (int l = 0; l < nl; ++l) m.kmax = m.k[l] > m.kmax ? m.k[l] : m.kmax;
    int32_t nq = 0;
    if (!rd(in, &nq, 1) || nq < 0) return 2;
    for (int i = 0; i < nq; ++i) {
        int32_t c[4];
        double lam[2];
        if (!rd(in, c, 4) || !rd(in, lam, 2)) return 2;
        if (c[0] < 0 || c[0] >= nl || c[2] < 0 || c[2] >= nl) return 2;
        const cd v = sigma_comp(m, mk(lam[0], lam[1]), c[0], c[1], c[2], c[3]);
        const double o[2] = {v.x, v.y};
        std::fwrite(o, sizeof(double), 2, out);
    }
    return 0;
}

static int run_bessel(FILE* in, FILE* out) {
    int32_t hdr[2];
    if (!rd(in, hdr, 2) || hdr[0] < 0 || hdr[1] < 0 || hdr[1] > 200) return 2;
    const int nx = hdr[0], p = hdr[1];
    std::vector<double> x(nx), J((size_t)nx * (p + 1));
    std::vector<cd> H((size_t)nx * (p + 1));
    if (!rd(in, x.data(), (size_t)nx)) return 2;
    for (int i = 0; i < nx; ++i) {
        bessel_j_seq(x[i], p, &J[(size_t)i * (p + 1)]);
        hankel_seq(x[i], p, &H[(size_t)i * (p + 1)]);
    }
    std::fwrite(J.data(), sizeof(double), J.size(), out);
    std::fwrite(H.data(), sizeof(cd), H.size(), out);
    return 0;
}

static int run_free(FILE* in, FILE* out) {
    int32_t nq = 0;
    if (!rd(in, &nq, 1) || nq < 0) return 2;
    for (int i = 0; i < nq; ++i) {
        double q[6];
        if (!rd(in, q, 6)) return 2;
        const cd v = free_kernel(q[0], q[1], q[2], q[3] != 0.0, q[4], q[5]);
        std::fwrite(&v, sizeof(cd), 1, out);
    }
    return 0;
}

static int run_self(FILE* in, FILE* out) {
    int32_t nq = 0;
    if (!rd(in, &nq, 1) || nq < 0) return 2;
    for (int i = 0; i < nq; ++i) {
        double q[3];
        if (!rd(in, q, 3)) return 2;
        const cd v = self_entry(q[0], q[1], q[2] != 0.0);
        std::fwrite(&v, sizeof(cd), 1, out);
    }
    return 0;
}

int main(int argc, char** argv) {
    if (argc != 4) {
        std::fprintf(stderr, "usage: devmath_harness sigma|bessel|free|self <input> <output>\n");
        return 2;
    }
    FILE* in = std::fopen(argv[2], "rb");
    FILE* out = std::fopen(argv[3], "wb");
    if (!in || !out) return 2;
    int rc = 2;
    if (std::strcmp(argv[1], "sigma") == 0) rc = run_sigma(in, out);
    else if (std::strcmp(argv[1], "bessel") == 0) rc = run_bessel(in, out);
    else if (std::strcmp(argv[1], "free") == 0) rc = run_free(in, out);
    else if (std::strcmp(argv[1], "self") == 0) rc = run_self(in, out);
    std::fclose(in);
    std::fclose(out);
    return rc;
}
