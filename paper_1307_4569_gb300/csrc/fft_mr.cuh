// Mixed-radix FFT with a compile-time radix list (lengths 2^a 3^b 5^c 7^d), the counterpart
// of fft_p2.cuh for the lattices whose FFT lengths are not powers of two.
//
// A transform of length N = R_0 R_1 ... R_{S-1} is computed by G threads (index t).  Stage s
// has N / R_s butterflies; butterfly j = t + G u (u < ceil(N / (R_s G)), j < N / R_s) of
// stage s is (Stockham, self-sorting):
//   inputs  x[j + r N/R_s],  twiddle exp(DIR 2 pi i r (j mod Ns) / (Ns R_s)),  DFT_{R_s},
//   outputs at (j div Ns) Ns R_s + (j mod Ns) + r Ns,        Ns = R_0 ... R_{s-1}.
// Stage 0 reads its inputs through the caller's load(e) functor; the last stage leaves its
// outputs in registers (register u R + r of thread t holds element t + G u + r N/R_last when
// t + G u < N/R_last: mr_out_pos / mr_out_ok); between stages the values cross one shared
// buffer, indexed through spad (one element of padding per 16), W transforms interleaved
// column-wise as in fft_p2.  Threads whose butterfly index passes N/R_s in a stage idle in it.
// In float the twiddle powers come from one first-order twiddle by a product tree (as in
// fft_p2); in double every power is read from the table tw[e] = exp(-2 pi i e / N).
#pragma once
#include "fft_p2.cuh"

namespace dgt {

// exp(DIR 2 pi i E / 9) times x, compile-time E in 1..8
template <int DIR, int E, typename C> __device__ __forceinline__ C w9(C x) {
    using R = typename RealOf<C>::type;
    constexpr double cs[9] = {1.0, 0.76604444311897803520, 0.17364817766693034885, -0.5, -0.93969262078590838405,
                              -0.93969262078590838405, -0.5, 0.17364817766693034885, 0.76604444311897803520};
    constexpr double sn[9] = {0.0, 0.64278760968653932632, 0.98480775301220805936, 0.86602540378443864676,
                              0.34202014332566873304, -0.34202014332566873304, -0.86602540378443864676,
                              -0.98480775301220805936, -0.64278760968653932632};
    return cmul(x, mk((R)cs[E], (R)(DIR * sn[E])));
}

// DFT_9 as 3 x 3: r = r1 + 3 r2, k = k1 + 3 k2; A[r1][k1] = DFT3_r2(v[r1 + 3 r2]) W9^{r1 k1},
// X[k1 + 3 k2] = DFT3_r1(A[r1][k1])
template <int DIR, typename C> __device__ __forceinline__ void dft9(C* v) {
    C a[3], b[3], c[3];
    a[0] = v[0]; a[1] = v[3]; a[2] = v[6];
    b[0] = v[1]; b[1] = v[4]; b[2] = v[7];
    c[0] = v[2]; c[1] = v[5]; c[2] = v[8];
    dft3<DIR>(a);
    dft3<DIR>(b);
    dft3<DIR>(c);
    b[1] = w9<DIR, 1>(b[1]); b[2] = w9<DIR, 2>(b[2]);
    c[1] = w9<DIR, 2>(c[1]); c[2] = w9<DIR, 4>(c[2]);
    C x0[3] = {a[0], b[0], c[0]}, x1[3] = {a[1], b[1], c[1]}, x2[3] = {a[2], b[2], c[2]};
    dft3<DIR>(x0);
    dft3<DIR>(x1);
    dft3<DIR>(x2);
#pragma unroll
    for (int k2 = 0; k2 < 3; ++k2) {
        v[0 + 3 * k2] = x0[k2];
        v[1 + 3 * k2] = x1[k2];
        v[2 + 3 * k2] = x2[k2];
    }
}

// DFT_15 by the prime-factor map (3 x 5, coprime, no twiddles): input r = (5 r1 + 3 r2) mod 15,
// output k = (10 k1 + 6 k2) mod 15 for k1 < 3, k2 < 5 (10 = 5 (5^-1 mod 3), 6 = 3 (3^-1 mod 5))
template <int DIR, typename C> __device__ __forceinline__ void dft15(C* v) {
    C a[5][3];
#pragma unroll
    for (int r2 = 0; r2 < 5; ++r2) {
#pragma unroll
        for (int r1 = 0; r1 < 3; ++r1) a[r2][r1] = v[(5 * r1 + 3 * r2) % 15];
        dft3<DIR>(a[r2]);
    }
    C o[15];
#pragma unroll
    for (int k1 = 0; k1 < 3; ++k1) {
        C b[5];
#pragma unroll
        for (int r2 = 0; r2 < 5; ++r2) b[r2] = a[r2][k1];
        dft5<DIR>(b);
#pragma unroll
        for (int k2 = 0; k2 < 5; ++k2) o[(10 * k1 + 6 * k2) % 15] = b[k2];
    }
#pragma unroll
    for (int i = 0; i < 15; ++i) v[i] = o[i];
}

template <int R, int DIR, bool PK, typename C> __device__ __forceinline__ void dft_mr(C* v) {
    if constexpr (R == 9) dft9<DIR>(v);
    else if constexpr (R == 15) dft15<DIR>(v);
    else dft_small<R, DIR, PK>(v);
}

template <int... Rs> struct RadixList {
    static constexpr int S = sizeof...(Rs);
    static constexpr int r[S] = {Rs...};
};

// F: the transform (N, G threads, radix list)
template <int N_, int G_, class RL> struct Mixed {
    static constexpr int N = N_;
    static constexpr int G = G_;
    static constexpr int NST = RL::S;
    static constexpr int radix(int s) { return RL::r[s]; }
    static constexpr int ns(int s) { return s == 0 ? 1 : ns(s - 1) * radix(s - 1); }
    static constexpr int nb(int s) { return N / radix(s); }
    static constexpr int bpt(int s) { return (nb(s) + G - 1) / G; }
    static constexpr int vals(int s) { return bpt(s) * radix(s); }
    static constexpr int vmax(int s) { return s == NST - 1 ? vals(s) : (vals(s) > vmax(s + 1) ? vals(s) : vmax(s + 1)); }
    static constexpr int V = vmax(0);                 // registers (complex values) per thread
    static constexpr int RL_ = radix(NST - 1);         // last radix
    static constexpr int NBL = nb(NST - 1);            // butterflies (and output stride) of the last stage
    static constexpr int OUT = vals(NST - 1);          // output registers
    static constexpr int SMEM = N + N / 16;            // padded elements per transform
    static_assert(ns(NST - 1) * radix(NST - 1) == N, "radices multiply to N");
};

// element held by output register idx of thread t, and whether it holds one
template <class F> __device__ __forceinline__ int mr_out_pos(int t, int idx) {
    return t + F::G * (idx / F::RL_) + (idx % F::RL_) * F::NBL;
}
template <class F> __device__ __forceinline__ bool mr_out_ok(int t, int idx) {
    return (F::NBL % F::G == 0) || t + F::G * (idx / F::RL_) < F::NBL;
}

template <class F, int DIR, int W, int S, bool PK, typename C>
__device__ __forceinline__ void mr_stages(int c, int t, C* sm, const C* __restrict__ tw, C (&v)[F::V]) {
    constexpr int Rp = F::radix(S - 1), Nsp = F::ns(S - 1), NBp = F::nb(S - 1), Bp = F::bpt(S - 1);
#pragma unroll
    for (int u = 0; u < Bp; ++u) {
        const int j = t + F::G * u;
        if (NBp % F::G == 0 || j < NBp) {
            const int base = (j / Nsp) * Nsp * Rp + (j % Nsp);
#pragma unroll
            for (int r = 0; r < Rp; ++r) sm[spad(base + r * Nsp) * W + c] = v[u * Rp + r];
        }
    }
    __syncthreads();
    constexpr int R = F::radix(S), Ns = F::ns(S), NB = F::nb(S), B = F::bpt(S);
    constexpr int TS = F::N / (Ns * R);
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int j = t + F::G * u;
        const bool on = NB % F::G == 0 || j < NB;
        const int jj = on ? j : 0;
        const int k = jj % Ns;
        if constexpr (sizeof(C) == 8) {
            C wp[R];
            wp[1] = __ldg(tw + k * TS);
            if (DIR > 0) wp[1].y = -wp[1].y;
#pragma unroll
            for (int r = 2; r < R; ++r) wp[r] = cmul(wp[r / 2], wp[r - r / 2]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const C x = sm[spad(jj + r * NB) * W + c];
                v[u * R + r] = r > 0 ? cmul(x, wp[r]) : x;
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C x = sm[spad(jj + r * NB) * W + c];
                if (r > 0) {
                    C w = __ldg(tw + r * k * TS);
                    if (DIR > 0) w.y = -w.y;
                    x = cmul(x, w);
                }
                v[u * R + r] = x;
            }
        }
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < B; ++u) dft_mr<R, DIR, PK>(v + u * R);
    if constexpr (S + 1 < F::NST) mr_stages<F, DIR, W, S + 1, PK>(c, t, sm, tw, v);
}

// Full transform: v receives the outputs (mr_out_pos / mr_out_ok).  All threads of the block
// call it (it synchronises the block); `sm` holds F::SMEM * W elements.
template <class F, int DIR, int W, bool PK = true, typename C, class Load>
__device__ __forceinline__ void fft_mr(int c, int t, C* sm, const C* __restrict__ tw, Load&& load, C (&v)[F::V]) {
    constexpr int R = F::radix(0), NB = F::nb(0), B = F::bpt(0);
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int j = t + F::G * u;
        const bool on = NB % F::G == 0 || j < NB;
#pragma unroll
        for (int r = 0; r < R; ++r) v[u * R + r] = on ? load(j + r * NB) : mk((typename RealOf<C>::type)0, (typename RealOf<C>::type)0);
    }
#pragma unroll
    for (int u = 0; u < B; ++u) dft_mr<R, DIR, PK>(v + u * R);
    if constexpr (F::NST > 1) mr_stages<F, DIR, W, 1, PK>(c, t, sm, tw, v);
}

}  // namespace dgt
