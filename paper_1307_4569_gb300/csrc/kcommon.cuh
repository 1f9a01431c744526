// Device helpers shared by the kernel translation units: chirp factors, typed loads and
// stores, and the output index map of the route post-processing.
#pragma once
#include "engine.h"

namespace dgt {

template <typename C> __device__ __forceinline__ C chirp_factor(const ChirpParams<C>& cp, int64_t l) {
    // pchirp(L, s)(l) = exp(pi i (s l^2 (L+1) mod 2L) / L) = exp(2 pi i e / 2L)
    const uint64_t twoL = 2 * (uint64_t)cp.L;
    const uint64_t lr = (uint64_t)l;
    const uint64_t l2 = (lr * lr) % twoL;
    const uint64_t t = mulmod(l2, ((uint64_t)cp.L + 1) % twoL, twoL);
    const uint64_t e = mulmod((uint64_t)cp.s_2L, t, twoL);
    C w = cp.cis2L((int64_t)e);
    if (cp.conj) w.y = -w.y;
    return w;
}

template <typename C> __device__ __forceinline__ C load_any(const void* p, int is_real, int64_t i) {
    using R = typename RealOf<C>::type;
    if (is_real) return mk(reinterpret_cast<const R*>(p)[i], (R)0);
    return reinterpret_cast<const C*>(p)[i];
}

template <typename C> __device__ __forceinline__ void store_any(void* p, int is_real, int64_t i, C v) {
    using R = typename RealOf<C>::type;
    if (is_real) reinterpret_cast<R*>(p)[i] = v.x;
    else reinterpret_cast<C*>(p)[i] = v;
}

// =====================================================================================
// output index map of one separable coefficient (analysis store / synthesis gather)
// row = (b, j, n) of Y, m = channel of the separable DGT.  Returns the offset into c
// and the phase to multiply with (analysis) -- synthesis uses its conjugate.
// =====================================================================================
template <typename C>
__device__ __forceinline__ int64_t out_index(const PostParams<C>& pp, const SepGeom& g, int64_t b, int64_t j,
                                             int64_t n, int64_t m, C& ph) {
    ph.x = 1;
    ph.y = 0;
    switch (pp.mode) {
        case POST_COSET: {
            const uint64_t e = mulmod((uint64_t)((n * pp.at) % pp.L), (uint64_t)__ldg(pp.sigma + j), (uint64_t)pp.L);
            ph = pp.cisL(-(int64_t)e);
            return (b * pp.N + pp.lam2 * n + j) * pp.M + m;
        }
        case POST_SHEAR0: {
            const uint64_t L = pp.L, twoN = 2 * (uint64_t)pp.N;
            const uint64_t sa = mulmod((uint64_t)pp.s1a_modL, (uint64_t)n, L);
            const int64_t rot = (int64_t)((L - sa) % L) / pp.b;
            const uint64_t nn = mulmod((uint64_t)n, (uint64_t)n, twoN);
            ph = pp.cis2N((int64_t)mulmod((uint64_t)pp.C1_2N, nn, twoN));
            int64_t mo = m + rot;
            if (mo >= pp.M) mo -= pp.M;
            return (b * pp.N + n) * pp.M + mo;
        }
        case POST_SHEAR1: {
            // separable channel kappa = m, separable time mr = n; Algorithm 1 index k = -kappa mod Nr
            const uint64_t N = pp.N, twoN = 2 * N, L = pp.L;
            const uint64_t k = (uint64_t)((pp.Nr - m) % pp.Nr);
            const uint64_t mr = (uint64_t)n;
            const uint64_t mt = (mulmod((uint64_t)pp.C1 % N, k % N, N) + mulmod((uint64_t)pp.C2_N, mr % N, N)) % N;
            const uint64_t sq1 = (mulmod((uint64_t)pp.C1_2N_, k % twoN, twoN) + mulmod((uint64_t)pp.C2_2N, mr % twoN, twoN)) % twoN;
            const uint64_t t1 = mulmod((uint64_t)pp.C3_2N, mulmod(sq1, sq1, twoN), twoN);
            const uint64_t inner = (mulmod((uint64_t)pp.C4_2N, mr % twoN, twoN) + mulmod((uint64_t)pp.C5_2N, k % twoN, twoN)) % twoN;
            const uint64_t t2 = mulmod(mr % twoN, inner, twoN);
            ph = pp.cis2N((int64_t)((t1 + twoN - t2) % twoN));
            const uint64_t kt = ((mulmod((uint64_t)pp.s1ar_L, k % L, L) + mulmod((uint64_t)pp.C6_L, mr % L, L)) % L) / (uint64_t)pp.b;
            return (b * pp.N + (int64_t)mt) * pp.M + (int64_t)kt;
        }
        default:
            return (b * g.d * g.q + n) * g.M + m;
    }
}

}  // namespace dgt
