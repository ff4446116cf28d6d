// Compile-time tables of the direct M2L's multiply-adds (Sec. 3: M2L as a sum over the parity
// window of Dt[o](k + b) Mt[t + o](b) for |k| + |b| <= rho), shared by the box form
// (translate.cu) and the occupied-cell form (m2l_sparse.cu).
#pragma once

#include "fc2t2_internal.cuh"

namespace fc2t2 {

// Cost of output k (the inputs b it takes) and the balanced split of the graded outputs into NS
// contiguous ranges: split s covers [dir_k0(s), dir_k0(s + 1)).
__host__ __device__ constexpr int dir_k0(int D, int rho, int NS, int s) {
    if (s <= 0) return 0;
    const int P = ncoef(D, rho);
    if (s >= NS) return P;
    long total = 0;
    for (int d = 0; d <= rho; ++d) total += (long)ncoef(D, d) * ncoef(D, rho - d) - (d ? (long)ncoef(D, d - 1) * ncoef(D, rho - d) : 0);
    // total = sum over k of ncoef(D, rho - |k|); cut where the running cost passes s / NS of it
    long run = 0;
    int k = 0;
    for (int d = 0; d <= rho; ++d) {
        const int cnt = ncoef(D, d) - (d ? ncoef(D, d - 1) : 0);
        for (int j = 0; j < cnt; ++j, ++k) {
            if (run * NS >= total * s) return k;
            run += ncoef(D, rho - d);
        }
    }
    return P;
}

// The (k, b) pairs of the outputs [K0, K1): every k in the range with every b, |k| + |b| <= RHO,
// ordered by b; entry = (k, b, index of k + b), all graded indices.  Built at compile time.
template <int D, int RHO, int K0, int K1>
struct DirPairs {
    static constexpr int count() {
        int c = 0;
        for (int bd = 0; bd <= RHO; ++bd)
            for (int b0 = bd; b0 >= 0; --b0)
                for (int b1 = bd - b0; b1 >= 0; --b1) {
                    if (D == 2 && bd - b0 - b1 != 0) continue;
                    for (int kd = 0; kd + bd <= RHO; ++kd)
                        for (int k0 = kd; k0 >= 0; --k0)
                            for (int k1 = kd - k0; k1 >= 0; --k1) {
                                if (D == 2 && kd - k0 - k1 != 0) continue;
                                const int ki = gidx<D>(k0, k1, kd - k0 - k1);
                                if (ki >= K0 && ki < K1) ++c;
                            }
                }
        return c;
    }
    static constexpr int N = count();
    short k[N > 0 ? N : 1], b[N > 0 ? N : 1], m[N > 0 ? N : 1];
    constexpr DirPairs() : k{}, b{}, m{} {
        int c = 0;
        for (int bd = 0; bd <= RHO; ++bd)
            for (int b0 = bd; b0 >= 0; --b0)
                for (int b1 = bd - b0; b1 >= 0; --b1) {
                    const int b2 = bd - b0 - b1;
                    if (D == 2 && b2 != 0) continue;
                    for (int kd = 0; kd + bd <= RHO; ++kd)
                        for (int k0 = kd; k0 >= 0; --k0)
                            for (int k1 = kd - k0; k1 >= 0; --k1) {
                                const int k2 = kd - k0 - k1;
                                if (D == 2 && k2 != 0) continue;
                                const int ki = gidx<D>(k0, k1, k2);
                                if (ki < K0 || ki >= K1) continue;
                                k[c] = (short)ki;
                                b[c] = (short)gidx<D>(b0, b1, b2);
                                m[c] = (short)gidx<D>(k0 + b0, k1 + b1, k2 + b2);
                                ++c;
                            }
                }
    }
};

}  // namespace fc2t2
