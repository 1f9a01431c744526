// Mixed-radix Stockham FFT on a shared-memory tile (radices 2, 3, 4, 5, 7, 8, 16).
//
// A CTA holds `nb` transforms of length n in shared memory; element (t, i) lives at
// buf[t * bs + i * es].  Stages alternate between two buffers of that layout (Stockham
// self-sorting form), so the result is in natural order.  Stage with radix R after
// radices of product Ns:
//   inputs  buf[j + r n/R],  twiddle exp(DIR 2 pi i r (j mod Ns) / (Ns R)),  DFT_R,
//   outputs buf[(j div Ns) Ns R + (j mod Ns) + r Ns].
// DIR = -1 is the forward transform sum_l x(l) e^{-2 pi i l k/n}; DIR = +1 the
// unnormalised inverse.  Twiddles come from a table tw[e] = exp(-2 pi i e / n) built on
// the host in double precision.
#pragma once
#include "cplx.cuh"

namespace dgt {

constexpr int kMaxStages = 24;

struct FftPlanDev {
    int n;
    int nst;
    int R[kMaxStages];
};

// ---------------------------------------------------------------------------------
// small DFTs in registers:  X[k] = sum_r x[r] exp(DIR 2 pi i r k / R)
// ---------------------------------------------------------------------------------
// PK = false keeps the float complex additions of the power-of-two codelets scalar (for a kernel
// that runs faster that way; the packed forms are the default)
template <bool PK, typename C> __device__ __forceinline__ C kadd(C a, C b) {
    if constexpr (PK) return cadd(a, b);
    a.x += b.x;
    a.y += b.y;
    return a;
}
template <bool PK, typename C> __device__ __forceinline__ C ksub(C a, C b) {
    if constexpr (PK) return csub(a, b);
    a.x -= b.x;
    a.y -= b.y;
    return a;
}

template <int DIR, bool PK = true, typename C> __device__ __forceinline__ void dft2(C& a, C& b) {
    C t = a;
    a = kadd<PK>(t, b);
    b = ksub<PK>(t, b);
}

template <int DIR, bool PK = true, typename C> __device__ __forceinline__ void dft4(C& x0, C& x1, C& x2, C& x3) {
    C s02 = kadd<PK>(x0, x2), d02 = ksub<PK>(x0, x2);
#ifdef DGT_PACKED_F32
    if constexpr (PK && sizeof(C) == 8) {
        const C s13 = cadd(x1, x3), d13 = csub(x1, x3);
        x0 = cadd(s02, s13);
        x2 = csub(s02, s13);
        x1 = cadd_ib<DIR>(d02, d13);
        x3 = cadd_ib<-DIR>(d02, d13);
        return;
    }
#endif
    C s13 = kadd<PK>(x1, x3), d13 = mul_i<DIR>(ksub<PK>(x1, x3));
    x0 = kadd<PK>(s02, s13);
    x2 = ksub<PK>(s02, s13);
    x1 = kadd<PK>(d02, d13);
    x3 = ksub<PK>(d02, d13);
}

// multiply by exp(DIR 2 pi i E / 16) for a compile-time E in 0..15
template <int DIR, int E, typename C> __device__ __forceinline__ C w16(C x) {
    using R = typename RealOf<C>::type;
    constexpr double c8 = 0.92387953251128675613, s8 = 0.38268343236508977173, h = 0.70710678118654752440;
    constexpr int e = E & 15;
    if constexpr (e == 0) {
        return x;
    } else if constexpr (e == 4) {
        return mul_i<DIR>(x);
    } else if constexpr (e >= 8) {
        C y = w16<DIR, e - 8>(x);
        return mk(-y.x, -y.y);
    } else {
        constexpr double cr = e == 1 ? c8 : e == 2 ? h : e == 3 ? s8 : e == 5 ? -s8 : e == 6 ? -h : -c8;
        constexpr double ci = e == 1 ? s8 : e == 2 ? h : e == 3 ? c8 : e == 5 ? c8 : e == 6 ? h : s8;
        C w = mk((R)cr, (R)(DIR * ci));
        return cmul(x, w);
    }
}

template <int DIR, bool PK = true, typename C> __device__ __forceinline__ void dft8(C* v) {
    // even/odd split: E = DFT4(v0,v2,v4,v6), O = DFT4(v1,v3,v5,v7), X[k] = E[k] + W8^k O[k]
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6];
    C o0 = v[1], o1 = v[3], o2 = v[5], o3 = v[7];
    dft4<DIR, PK>(e0, e1, e2, e3);
    dft4<DIR, PK>(o0, o1, o2, o3);
    o1 = w16<DIR, 2>(o1);
    o2 = w16<DIR, 4>(o2);
    o3 = w16<DIR, 6>(o3);
    v[0] = kadd<PK>(e0, o0); v[4] = ksub<PK>(e0, o0);
    v[1] = kadd<PK>(e1, o1); v[5] = ksub<PK>(e1, o1);
    v[2] = kadd<PK>(e2, o2); v[6] = ksub<PK>(e2, o2);
    v[3] = kadd<PK>(e3, o3); v[7] = ksub<PK>(e3, o3);
}

template <int DIR, bool PK = true, typename C> __device__ __forceinline__ void dft16(C* v) {
    // r = r1 + 4 r2, k = k1 + 4 k2:  A[r1][k1] = DFT4_r2(v[r1 + 4 r2]) W16^{r1 k1},
    // X[k1 + 4 k2] = DFT4_r1(A[r1][k1])
    dft4<DIR, PK>(v[0], v[4], v[8], v[12]);
    dft4<DIR, PK>(v[1], v[5], v[9], v[13]);
    dft4<DIR, PK>(v[2], v[6], v[10], v[14]);
    dft4<DIR, PK>(v[3], v[7], v[11], v[15]);
    // A[r1][k1] now sits at v[r1 + 4 k1]
    v[5] = w16<DIR, 1>(v[5]);   v[9] = w16<DIR, 2>(v[9]);   v[13] = w16<DIR, 3>(v[13]);
    v[6] = w16<DIR, 2>(v[6]);   v[10] = w16<DIR, 4>(v[10]); v[14] = w16<DIR, 6>(v[14]);
    v[7] = w16<DIR, 3>(v[7]);   v[11] = w16<DIR, 6>(v[11]); v[15] = w16<DIR, 9>(v[15]);
    dft4<DIR, PK>(v[0], v[1], v[2], v[3]);
    dft4<DIR, PK>(v[4], v[5], v[6], v[7]);
    dft4<DIR, PK>(v[8], v[9], v[10], v[11]);
    dft4<DIR, PK>(v[12], v[13], v[14], v[15]);
    // X[k1 + 4 k2] sits at v[4 k1 + k2]: transpose the 4x4 index
    C t;
    t = v[1]; v[1] = v[4]; v[4] = t;
    t = v[2]; v[2] = v[8]; v[8] = t;
    t = v[3]; v[3] = v[12]; v[12] = t;
    t = v[6]; v[6] = v[9]; v[9] = t;
    t = v[7]; v[7] = v[13]; v[13] = t;
    t = v[11]; v[11] = v[14]; v[14] = t;
}

template <int DIR, typename C> __device__ __forceinline__ void dft3(C* v) {
    using R = typename RealOf<C>::type;
    constexpr double s3 = 0.86602540378443864676;
    C t = cadd(v[1], v[2]);
    C u = mul_i<DIR>(cscale(csub(v[1], v[2]), (R)s3));
    C m = csub(v[0], cscale(t, (R)0.5));
    v[0] = cadd(v[0], t);
    v[1] = cadd(m, u);
    v[2] = csub(m, u);
}

template <int DIR, typename C> __device__ __forceinline__ void dft5(C* v) {
    using R = typename RealOf<C>::type;
    constexpr double c1 = 0.30901699437494742410, c2 = -0.80901699437494742410;
    constexpr double s1 = 0.95105651629515357212, s2 = 0.58778525229247312917;
    C t1 = cadd(v[1], v[4]), t2 = cadd(v[2], v[3]);
    C t3 = csub(v[1], v[4]), t4 = csub(v[2], v[3]);
    C x0 = v[0];
    C a1 = cadd(x0, cadd(cscale(t1, (R)c1), cscale(t2, (R)c2)));
    C a2 = cadd(x0, cadd(cscale(t1, (R)c2), cscale(t2, (R)c1)));
    C b1 = mul_i<DIR>(cadd(cscale(t3, (R)s1), cscale(t4, (R)s2)));
    C b2 = mul_i<DIR>(csub(cscale(t3, (R)s2), cscale(t4, (R)s1)));
    v[0] = cadd(x0, cadd(t1, t2));
    v[1] = cadd(a1, b1);
    v[4] = csub(a1, b1);
    v[2] = cadd(a2, b2);
    v[3] = csub(a2, b2);
}

template <int DIR, typename C> __device__ __forceinline__ void dft7(C* v) {
    using R = typename RealOf<C>::type;
    constexpr double cs[4] = {1.0, 0.62348980185873353053, -0.22252093395631440429, -0.90096886790241912624};
    constexpr double sn[4] = {0.0, 0.78183148246802980871, 0.97492791218182360702, 0.43388373911755812048};
    C t[4], u[4];
#pragma unroll
    for (int k = 1; k <= 3; ++k) {
        t[k] = cadd(v[k], v[7 - k]);
        u[k] = csub(v[k], v[7 - k]);
    }
    C x0 = v[0];
    v[0] = cadd(x0, cadd(t[1], cadd(t[2], t[3])));
#pragma unroll
    for (int j = 1; j <= 3; ++j) {
        C A = x0, B = mk((R)0, (R)0);
#pragma unroll
        for (int k = 1; k <= 3; ++k) {
            const int e = (j * k) % 7;                 // cos(2 pi e/7), sin(2 pi e/7)
            const int ee = e <= 3 ? e : 7 - e;
            const double sg = e <= 3 ? 1.0 : -1.0;
            A = cadd(A, cscale(t[k], (R)cs[ee]));
            B = cadd(B, cscale(u[k], (R)(sg * sn[ee])));
        }
        B = mul_i<DIR>(B);
        v[j] = cadd(A, B);
        v[7 - j] = csub(A, B);
    }
}

template <int R, int DIR, bool PK = true, typename C> __device__ __forceinline__ void dft_small(C* v) {
    if constexpr (R == 2) dft2<DIR, PK>(v[0], v[1]);
    else if constexpr (R == 3) dft3<DIR>(v);
    else if constexpr (R == 4) dft4<DIR, PK>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 5) dft5<DIR>(v);
    else if constexpr (R == 7) dft7<DIR>(v);
    else if constexpr (R == 8) dft8<DIR, PK>(v);
    else if constexpr (R == 16) dft16<DIR, PK>(v);
}

// ---------------------------------------------------------------------------------
// one Stockham stage, out of place (src -> dst), over all nb transforms of the tile.
// BATCH_FAST: consecutive threads take consecutive transforms t (interleaved layouts,
// bs == 1); otherwise consecutive butterflies j of one transform (row layouts, es == 1).
// Each butterfly is loaded, transformed and stored at once: only R values are live.
// ---------------------------------------------------------------------------------
template <int R, int DIR, bool BATCH_FAST, typename C>
__device__ __forceinline__ void stockham_stage(const C* __restrict__ src, C* __restrict__ dst, int n, int nb, int es,
                                               int bs, int Ns, const C* __restrict__ tw) {
    const int nbf = n / R;
    const int tstride = n / (Ns * R);
    // butterfly (t, j), j = jq Ns + k: the thread's first index is split once with divisions,
    // then advanced by the block size with adds and carries only (nbf is a multiple of Ns)
    const int T = blockDim.x;
    const int idx0 = threadIdx.x;
    int t, j;
    int dt, dj;                              // the block step split like an index
    if (BATCH_FAST) {
        t = idx0 % nb; j = idx0 / nb;
        dt = T % nb; dj = T / nb;
    } else {
        j = idx0 % nbf; t = idx0 / nbf;
        dj = T % nbf; dt = T / nbf;
    }
    int jq = j / Ns, k = j - jq * Ns;
    const int djq = dj / Ns, dk = dj - djq * Ns;
    const int nq = nbf / Ns;
    for (; BATCH_FAST ? j < nbf : t < nb;) {
        const C* s = src + t * bs;
        C* d = dst + t * bs;
        C v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            C x = s[(j + r * nbf) * es];
            if (r > 0 && k > 0) {
                C w = __ldg(tw + r * k * tstride);
                if (DIR > 0) w.y = -w.y;
                x = cmul(x, w);
            }
            v[r] = x;
        }
        dft_small<R, DIR>(v);
        const int base = jq * Ns * R + k;
#pragma unroll
        for (int r = 0; r < R; ++r) d[(base + r * Ns) * es] = v[r];
        // advance (t, j) by T
        if (BATCH_FAST) {
            t += dt;
            j += dj; jq += djq; k += dk;
            if (t >= nb) { t -= nb; ++j; ++k; }
        } else {
            j += dj; jq += djq; k += dk;
            t += dt;
            if (j >= nbf) { j -= nbf; jq -= nq; ++t; }
        }
        if (k >= Ns) { k -= Ns; ++jq; }
    }
}

// Full transform of the tile held in buffer `a` (same layout in the spare buffer `b`).
// The caller synchronises the block before the call; the function ends synchronised and
// returns the buffer that holds the result (a or b, by the parity of the stage count).
template <int DIR, bool BATCH_FAST, typename C>
__device__ C* fft_tile(C* a, C* b, const FftPlanDev& pl, int nb, int es, int bs, const C* __restrict__ tw) {
    C* src = a;
    C* dst = b;
    int Ns = 1;
    for (int st = 0; st < pl.nst; ++st) {
        const int R = pl.R[st];
        switch (R) {
            case 16: stockham_stage<16, DIR, BATCH_FAST>(src, dst, pl.n, nb, es, bs, Ns, tw); break;
            case 8: stockham_stage<8, DIR, BATCH_FAST>(src, dst, pl.n, nb, es, bs, Ns, tw); break;
            case 4: stockham_stage<4, DIR, BATCH_FAST>(src, dst, pl.n, nb, es, bs, Ns, tw); break;
            case 2: stockham_stage<2, DIR, BATCH_FAST>(src, dst, pl.n, nb, es, bs, Ns, tw); break;
            case 3: stockham_stage<3, DIR, BATCH_FAST>(src, dst, pl.n, nb, es, bs, Ns, tw); break;
            case 5: stockham_stage<5, DIR, BATCH_FAST>(src, dst, pl.n, nb, es, bs, Ns, tw); break;
            case 7: stockham_stage<7, DIR, BATCH_FAST>(src, dst, pl.n, nb, es, bs, Ns, tw); break;
            default: break;
        }
        __syncthreads();
        C* t = src;
        src = dst;
        dst = t;
        Ns *= R;
    }
    return src;
}

}  // namespace dgt
