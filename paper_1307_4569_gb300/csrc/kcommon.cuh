// Device helpers shared by the kernel translation units: chirp factors, typed loads and
// stores, and the output index map of the route post-processing.
#pragma once
#include "engine.h"

namespace dgt {

// pchirp(L, s)(l) = exp(pi i (s l^2 (L+1) mod 2L) / L) = exp(2 pi i e / 2L), 0 <= l < L, from
// the exact integer exponent (three reductions modulo 2L and a two-level table lookup)
template <typename C> __device__ __forceinline__ C chirp_exact(const ChirpParams<C>& cp, int64_t l) {
    const uint64_t lr = (uint64_t)l;
    const uint64_t l2 = cp.m2L.mod(lr * lr);
    const uint64_t t = cp.m2L.mulmod(l2, (uint64_t)cp.L + 1);
    const uint64_t e = cp.m2L.mulmod((uint64_t)cp.s_2L, t);
    C w = cp.cis2L.at(e);
    if (cp.conj) w.y = -w.y;
    return w;
}

// the chirp factor of sample l < L: one load from the plan's table of chirp_exact's values
// (bit-identical) when it has one, else computed
template <typename C> __device__ __forceinline__ C chirp_factor(const ChirpParams<C>& cp, int64_t l) {
    if (cp.tab) {
        C w = __ldg(cp.tab + l);
        if (cp.conj) w.y = -w.y;
        return w;
    }
    return chirp_exact(cp, l);
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
            // n * at < L and sigma_j < b <= L
            const uint64_t e = pp.mL.mulmod((uint64_t)(n * pp.at), (uint64_t)__ldg(pp.sigma + j));
            ph = pp.cisL.at(e ? (uint64_t)pp.L - e : 0);
            return (b * pp.N + pp.lam2 * n + j) * pp.M + m;
        }
        case POST_SHEAR0: {
            const uint64_t L = pp.L;
            const uint64_t sa = pp.mL.mulmod((uint64_t)pp.s1a_modL, (uint64_t)n);
            const int64_t rot = (int64_t)pp.mb.div(sa ? L - sa : 0);
            const uint64_t nn = pp.m2N.mulmod((uint64_t)n, (uint64_t)n);
            ph = pp.cis2N.at(pp.m2N.mulmod((uint64_t)pp.C1_2N, nn));
            int64_t mo = m + rot;
            if (mo >= pp.M) mo -= pp.M;
            return (b * pp.N + n) * pp.M + mo;
        }
        case POST_SHEAR1: {
            // separable channel kappa = m, separable time mr = n; Algorithm 1 index k = -kappa mod Nr
            const uint64_t twoN = 2 * (uint64_t)pp.N, L = pp.L;
            const uint64_t k = m ? (uint64_t)(pp.Nr - m) : 0;
            const uint64_t mr = (uint64_t)n;
            const uint64_t k2 = pp.m2N.mod(k), mr2 = pp.m2N.mod(mr);
            const uint64_t sq1 = pp.m2N.mod(pp.m2N.mulmod((uint64_t)pp.C1_2N_, k2) + pp.m2N.mulmod((uint64_t)pp.C2_2N, mr2));
            const uint64_t mt = pp.mN.mod(sq1);
            const uint64_t t1 = pp.m2N.mulmod((uint64_t)pp.C3_2N, pp.m2N.mulmod(sq1, sq1));
            const uint64_t inner = pp.m2N.mod(pp.m2N.mulmod((uint64_t)pp.C4_2N, mr2) + pp.m2N.mulmod((uint64_t)pp.C5_2N, k2));
            const uint64_t t2 = pp.m2N.mulmod(mr2, inner);
            ph = pp.cis2N.at(t1 >= t2 ? t1 - t2 : t1 + twoN - t2);
            const uint64_t kt = pp.mb.div(pp.mL.mod(pp.mL.mulmod((uint64_t)pp.s1ar_L, pp.mL.mod(k)) +
                                                    pp.mL.mulmod((uint64_t)pp.C6_L, pp.mL.mod(mr))));
            return (b * pp.N + (int64_t)mt) * pp.M + (int64_t)kt;
        }
        default:
            return (b * g.d * g.q + n) * g.M + m;
    }
}

// The frequency-shear map (POST_SHEAR1) of one row in 32-bit arithmetic: the terms that
// depend on the separable time index n alone are formed once per row, the rest per channel.
// Same values as out_index (sh1_fast rows only).
struct Sh1Row {
    uint32_t A;        // C2 n mod 2N
    uint32_t Bq;       // C4 n mod 2N
    uint32_t Kc;       // C6 n mod L
    uint32_t n2;       // n mod 2N
    uint32_t al, be;   // n2 Bq and n2 C5 mod 2N: the phase term n2 (Bq + C5 k) = al + be k
    int64_t base;      // b N M
};
template <typename C> __device__ __forceinline__ Sh1Row sh1_row(const PostParams<C>& pp, int64_t b, int64_t n) {
    Sh1Row r;
    r.n2 = pp.q2N.mod((uint32_t)n);
    r.A = pp.q2N.mod(pp.f_C2 * r.n2);
    r.Bq = pp.q2N.mod(pp.f_C4 * r.n2);
    r.Kc = pp.qL.mod((uint32_t)((uint64_t)pp.f_C6 * (uint32_t)n % pp.qL.d));
    r.al = pp.q2N.mod(r.n2 * r.Bq);
    r.be = pp.q2N.mod(r.n2 * pp.f_C5);
    r.base = b * pp.N * pp.M;
    return r;
}
// the output time mt and channel kt of channel m of the row (the coefficient's offset is
// base + mt M + kt), and the exponent e of its phase exp(2 pi i e / 2N) (pp.cis2N.at(e))
template <typename C>
__device__ __forceinline__ void sh1_index(const PostParams<C>& pp, const Sh1Row& r, int m, uint32_t& e, uint32_t& mt,
                                          uint32_t& kt) {
    const uint32_t twoN = pp.q2N.d;
    const uint32_t k = m ? pp.f_Nr - (uint32_t)m : 0u;           // -kappa mod Nr
    const uint32_t k2 = pp.q2N.mod(k);
    const uint32_t sq1 = pp.q2N.mod(pp.f_C1 * k2 + r.A);
    mt = sq1 >= pp.f_N ? sq1 - pp.f_N : sq1;
    const uint32_t t1 = pp.q2N.mod(pp.f_C3 * pp.q2N.mod(sq1 * sq1));
    const uint32_t inner = pp.q2N.mod(r.Bq + pp.f_C5 * k2);
    const uint32_t t2 = pp.q2N.mod(r.n2 * inner);
    e = t1 >= t2 ? t1 - t2 : t1 + twoN - t2;
    kt = pp.qb.div(pp.qL.mod(pp.f_s1ar * pp.qL.mod(k) + r.Kc));
}
// sh1_index for the rows whose output channel is known (s1 = 0: the tile kernels): the time mt
// and the phase exponent e only, with k < Nr <= N < 2N its own residue, and the quadratic term
// skipped when C3 = 0 (same values)
template <typename C>
__device__ __forceinline__ void sh1_index_t(const PostParams<C>& pp, const Sh1Row& r, int m, uint32_t& e,
                                            uint32_t& mt) {
    const uint32_t twoN = pp.q2N.d;
    const uint32_t k = m ? pp.f_Nr - (uint32_t)m : 0u;
    const uint32_t sq1 = pp.q2N.mod(pp.f_C1 * k + r.A);
    mt = sq1 >= pp.f_N ? sq1 - pp.f_N : sq1;
    const uint32_t t1 = pp.f_C3 ? pp.q2N.mod(pp.f_C3 * pp.q2N.mod(sq1 * sq1)) : 0u;
    const uint32_t t2 = pp.q2N.mod(r.al + r.be * k);
    e = t1 >= t2 ? t1 - t2 : t1 + twoN - t2;
}
template <typename C>
__device__ __forceinline__ void sh1_split(const PostParams<C>& pp, const Sh1Row& r, int m, C& ph, uint32_t& mt,
                                          uint32_t& kt) {
    uint32_t e;
    sh1_index(pp, r, m, e, mt, kt);
    ph = pp.cis2N.at(e);
}
template <typename C>
__device__ __forceinline__ int64_t sh1_at(const PostParams<C>& pp, const Sh1Row& r, int m, C& ph) {
    uint32_t mt, kt;
    sh1_split(pp, r, m, ph, mt, kt);
    return r.base + (int64_t)mt * pp.M + kt;
}

}  // namespace dgt
