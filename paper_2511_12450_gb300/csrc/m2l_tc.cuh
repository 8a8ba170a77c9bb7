// m2l_tc.cuh -- block right-hand-side M2L of the precision form on the tensor
// cores (tcgen05, kind::tf32).  Included by mixed.cu after its FP32 helpers.
//
// With many right-hand sides (incidence angles, Sec. 5 Examples 2-3) the M2L of a
// target box is a sum of dense products: for each list entry e,
//   out_dst(e) += A_e X_S(e),
// A_e the entry's (2p+1) x (2p+1) scaled FP32 translation (the free-space Graf
// table, or the reaction moment table of eq. generalintegral with the departure
// and arrival flips and the mirror symmetry folded in) and X_S the (2p+1) x ncols
// block of the source's scaled multipoles.  Complex products in real form,
//   [Re Y; Im Y] = [[Ar, -Ai], [Ai, Ar]] [Re X; Im X],
// so one MMA has M = 128 >= 2(2p+1) rows, K = 2 kh padded to a multiple of 8 (the real
// part's columns from K = 0, the imaginary part's from kh = 2p+1 rounded up to 4, so that
// staging writes 16-byte row segments),
// and N = the columns padded to a multiple of 16 (at most TC_MAXN per launch).
// Every operand is split into a TF32 head and an FP32 tail, and the three
// products head.head + head.tail + tail.head (3xTF32) keep the FP32 accuracy of
// the SIMT kernel.
//
// One CTA (4 warps) per target box.  Per entry all threads stage A_e and X_S into
// shared memory in the K-major no-swizzle canonical layout (core matrices of 8
// rows x 16 bytes, contiguous along K, 8-row groups kp/4 core matrices apart);
// one thread issues the entry's chain of tcgen05.mma into a TMEM accumulator and
// tcgen05.commit arrives on an mbarrier, which every thread waits on (bounded).
// Each warp then reads its 32 rows of the product with tcgen05.ld and adds them
// to register sums for the entry's output (cell centre or one of the two
// reaction centres).  The tensor cores thus accumulate one entry's 3 x kp/8 MMAs
// only: accumulating a whole box (~40 entries) in TMEM lost about 5e-6 relative,
// their accumulation drifting faster than round-to-nearest FP32, while the
// per-entry register sums keep about 4e-7.  At the end row r < 2p+1 holds real
// parts, the next 2p+1 rows imaginary parts.  If a wait gives up, the box's
// outputs are written as zeros and *err is set (the host reports it).
#pragma once

#define TC_MAXN 32          // columns per launch (N of the MMA)
#define TC_UNITS 4          // staging units (4 table values each) loaded together
#define TC_WAIT_LIMIT (1 << 24)

__device__ __forceinline__ uint32_t tc_smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// float index of element (row, k) of a K-major canonical operand with kp columns
__device__ __forceinline__ int tc_canon(int row, int k, int kp) {
    return (((row >> 3) * (kp >> 2) + (k >> 2)) << 5) + ((row & 7) << 2) + (k & 3);
}

// shared-memory matrix descriptor: start address, leading (K) core-matrix stride
// 128 B, stride between 8-row groups sbo, descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr, uint32_t sbo) {
    return (uint64_t)((saddr & 0x3FFFF) >> 4) | ((uint64_t)(128 >> 4) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// a = head + tail, head = a rounded to TF32 (low 13 mantissa bits zero)
__device__ __forceinline__ void tc_split(float a, float& hi, float& lo) {
    uint32_t h;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(h) : "f"(a));
    hi = __uint_as_float(h);
    lo = a - hi;
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                 "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
                 ::"r"(d), "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ bool tc_wait(uint32_t mbar, uint32_t parity) {
    uint32_t done = 0;
    for (int it = 0; it < TC_WAIT_LIMIT && !done; ++it)
        asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done) : "r"(mbar), "r"(parity));
    return done != 0;
}

// value of the entry's translation at (output i, source coefficient j), both 0..2p
__device__ __forceinline__ cf tc_entry_value(const M2LEnt& E, int i, int j, int p, int nco,
                                            const cf* __restrict__ ftab, const int64_t* __restrict__ ftab_off,
                                            const cf* __restrict__ rtab) {
    if (!(E.flags & M2L_REACT)) return ftab[ftab_off[E.tab] + (int64_t)j * nco + i];   // (n_out, m_in) column-major
    const bool bdown = (E.flags & M2L_B_DOWN) != 0;
    const int nn = i - p, mrow = bdown ? nn : -nn;
    const bool adown = (E.flags & M2L_A_DOWN) != 0;
    const int mi = adown ? j : 2 * p - j;   // departure up: alpha_n = (-1)^n M_{-n}
    // a mirrored table is read at (-mrow, -n)
    const cf v = (E.flags & M2L_FLIP) ? rtab[E.tab + (p - mrow) + (int64_t)(2 * p - mi) * nco]
                                      : rtab[E.tab + (mrow + p) + (int64_t)mi * nco];
    const bool neg = ((!bdown) && (mrow & 1)) != ((!adown) && ((p - j) & 1));
    return neg ? mkf(-v.x, -v.y) : v;
}

template <int NP>
__global__ void __launch_bounds__(128) k_m2l32_tc(
    const int* __restrict__ boxes, const int* __restrict__ ent_ptr, const M2LEnt* __restrict__ ents,
    const int* __restrict__ box_level, const int* __restrict__ p_level, const int64_t* __restrict__ coef_off,
    const int* __restrict__ slot_of, const int64_t* __restrict__ slot_coef, const cf* __restrict__ ftab,
    const int64_t* __restrict__ ftab_off, const cf* __restrict__ rtab, int col0, int ncols, int kp,
    int64_t ncoef, int64_t nslotcoef, const cf* __restrict__ Min, const cf* __restrict__ Mp,
    cf* __restrict__ Lout, cf* __restrict__ Lp, int* __restrict__ err) {
    constexpr uint32_t TCOLS = 32;   // TMEM columns: one NP-wide accumulator
    extern __shared__ __align__(1024) float tsm[];
    float* sAh = tsm;
    float* sAl = sAh + 128 * kp;
    float* sBh = sAl + 128 * kp;
    float* sBl = sBh + NP * kp;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int T = boxes[blockIdx.x];
    const int p = p_level[box_level[T]], nco = 2 * p + 1, n2 = 2 * nco;
    const int e0 = ent_ptr[T], e1 = ent_ptr[T + 1];
    const uint32_t mb = tc_smem_addr(&mbar);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(tc_smem_addr(&tmem_base)),
                     "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(mb));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    // zero the operand buffers once: the padding rows and columns stay zero
    for (int i = tid; i < (2 * 128 + 2 * NP) * kp; i += 128) tsm[i] = 0.f;
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tb = tmem_base;
    const uint32_t trow = tb + ((uint32_t)(warp * 32) << 16);   // this warp's 32 lanes
    // D F32 (bits 4-5), A and B TF32 (7-9, 10-12), both K-major, N >> 3 (17-22), M >> 4 (24-28)
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NP >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
    const uint32_t sbo = (uint32_t)(kp >> 2) * 128;
    float acc0[NP], acc1[NP], acc2[NP];
#pragma unroll
    for (int c = 0; c < NP; ++c) { acc0[c] = 0.f; acc1[c] = 0.f; acc2[c] = 0.f; }
    uint32_t phase = 0;
    bool ok = true;
    for (int e = e0; e < e1 && ok; ++e) {
        const M2LEnt E = ents[e];
        // four consecutive K positions per store (one 16-byte row segment of a core matrix):
        // the real part's columns start at K = 0, the imaginary part's at K = kh (a multiple of
        // four), the positions between nco and kh are written as zeros
        const int kh = (nco + 3) & ~3, nq = kh >> 2;
        // TC_UNITS units per round: all their table values are loaded before any is split or
        // stored, so their loads are in flight together
        for (int q0 = tid; q0 < nco * nq; q0 += 128 * TC_UNITS) {
            cf raw[TC_UNITS][4];
#pragma unroll
            for (int u = 0; u < TC_UNITS; ++u) {
                const int q = q0 + 128 * u;
                const int i = q % nco, j0 = (q / nco) * 4;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    raw[u][t] = (q < nco * nq && j0 + t < nco) ? tc_entry_value(E, i, j0 + t, p, nco, ftab, ftab_off, rtab)
                                                             : mkf(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < TC_UNITS; ++u) {
                const int q = q0 + 128 * u;
                if (q >= nco * nq) break;
                const int i = q % nco, j0 = (q / nco) * 4;
                float4 arh, arl, aih, ail;
                float* f[4] = {&arh.x, &arl.x, &aih.x, &ail.x};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    tc_split(raw[u][t].x, f[0][t], f[1][t]);
                    tc_split(raw[u][t].y, f[2][t], f[3][t]);
                }
                const float4 naih = make_float4(-aih.x, -aih.y, -aih.z, -aih.w);
                const float4 nail = make_float4(-ail.x, -ail.y, -ail.z, -ail.w);
                *(float4*)&sAh[tc_canon(i, j0, kp)] = arh;            *(float4*)&sAl[tc_canon(i, j0, kp)] = arl;
                *(float4*)&sAh[tc_canon(i, kh + j0, kp)] = naih;      *(float4*)&sAl[tc_canon(i, kh + j0, kp)] = nail;
                *(float4*)&sAh[tc_canon(i + nco, j0, kp)] = aih;      *(float4*)&sAl[tc_canon(i + nco, j0, kp)] = ail;
                *(float4*)&sAh[tc_canon(i + nco, kh + j0, kp)] = arh; *(float4*)&sAl[tc_canon(i + nco, kh + j0, kp)] = arl;
            }
        }
        const bool from_slot = (E.flags & M2L_REACT) && (E.flags & M2L_SRC_SLOT);
        const cf* src = (from_slot ? Mp : Min) + E.src;
        const int64_t stride = from_slot ? nslotcoef : ncoef;
        for (int q0 = tid; q0 < ncols * nq; q0 += 128 * TC_UNITS) {
            cf raw[TC_UNITS][4];
#pragma unroll
            for (int u = 0; u < TC_UNITS; ++u) {
                const int q = q0 + 128 * u;
                const int jq = q % nq, c = q / nq, j0 = jq * 4;
#pragma unroll
                for (int t = 0; t < 4; ++t)
                    raw[u][t] = (q < ncols * nq && j0 + t < nco) ? src[(int64_t)(col0 + c) * stride + j0 + t]
                                                                 : mkf(0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < TC_UNITS; ++u) {
                const int q = q0 + 128 * u;
                if (q >= ncols * nq) break;
                const int jq = q % nq, c = q / nq, j0 = jq * 4;
                float4 xrh, xrl, xih, xil;
                float* f[4] = {&xrh.x, &xrl.x, &xih.x, &xil.x};
#pragma unroll
                for (int t = 0; t < 4; ++t) {
                    tc_split(raw[u][t].x, f[0][t], f[1][t]);
                    tc_split(raw[u][t].y, f[2][t], f[3][t]);
                }
                *(float4*)&sBh[tc_canon(c, j0, kp)] = xrh;       *(float4*)&sBl[tc_canon(c, j0, kp)] = xrl;
                *(float4*)&sBh[tc_canon(c, kh + j0, kp)] = xih;  *(float4*)&sBl[tc_canon(c, kh + j0, kp)] = xil;
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (tid == 0) {
            const uint32_t ah = tc_smem_addr(sAh), al = tc_smem_addr(sAl);
            const uint32_t bh = tc_smem_addr(sBh), bl = tc_smem_addr(sBl);
            for (int ks = 0; ks < kp / 8; ++ks) {
                const uint32_t o = (uint32_t)ks * 256;
                tc_mma(tb, tc_desc(ah + o, sbo), tc_desc(bh + o, sbo), idesc, ks > 0 ? 1u : 0u);
                tc_mma(tb, tc_desc(ah + o, sbo), tc_desc(bl + o, sbo), idesc, 1u);
                tc_mma(tb, tc_desc(al + o, sbo), tc_desc(bh + o, sbo), idesc, 1u);
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mb));
        }
        const bool done = tc_wait(mb, phase);
        ok = __syncthreads_and(done) != 0;
        if (!ok) { tc_wait(mb, phase); break; }   // the chain in flight, once more (bounded), before the TMEM is freed
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;");
        const int dst = (E.flags & M2L_REACT) ? (E.flags >> M2L_DST_SHIFT) & 3 : 0;
#pragma unroll
        for (int c0 = 0; c0 < NP; c0 += 16) {
            uint32_t r[16];
            asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                         : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                           "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                           "=r"(r[14]), "=r"(r[15])
                         : "r"(trow + (uint32_t)c0));
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            if (dst == 0) {
#pragma unroll
                for (int c = 0; c < 16; ++c) acc0[c0 + c] += __uint_as_float(r[c]);
            } else if (dst == 1) {
#pragma unroll
                for (int c = 0; c < 16; ++c) acc1[c0 + c] += __uint_as_float(r[c]);
            } else {
#pragma unroll
                for (int c = 0; c < 16; ++c) acc2[c0 + c] += __uint_as_float(r[c]);
            }
        }
        asm volatile("tcgen05.fence::before_thread_sync;");
    }
    if (!ok && tid == 0) atomicExch(err, 1);
    const int row = warp * 32 + lane;
    if (row < n2) {
        const int i = row < nco ? row : row - nco;
        const int part = row < nco ? 0 : 1;
        for (int dst = 0; dst < 3; ++dst) {
            cf* out;
            int64_t base, ostride;
            if (dst == 0) {
                out = Lout; base = coef_off[T]; ostride = ncoef;
            } else {
                const int ts = slot_of[2 * T + dst - 1];
                if (ts < 0) continue;
                out = Lp; base = slot_coef[ts]; ostride = nslotcoef;
            }
#pragma unroll
            for (int c = 0; c < NP; ++c) {
                const float v = !ok ? 0.f : (dst == 0 ? acc0[c] : dst == 1 ? acc1[c] : acc2[c]);
                if (c < ncols) ((float*)(out + (int64_t)(col0 + c) * ostride + base + i))[part] = v;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tb), "r"(TCOLS));
}
