// Power-of-two FFT with compile-time length N (16 <= N <= 16384), 16 values per thread.
//
// A transform is computed by G = N/16 threads (index t).  Stage s has radix R_s = 16, except
// the last stage whose radix is 2^(log2 N mod 4) when that is not 0; each thread performs
// 16/R_s butterflies j = t + G u of the stage (Stockham, self-sorting):
//   inputs  x[j + r N/R],  twiddle exp(DIR 2 pi i r (j mod Ns)/(Ns R)),  DFT_R,
//   outputs at (j div Ns) Ns R + (j mod Ns) + r Ns,          Ns = product of earlier radices.
// Stage 0 reads its inputs through the caller's load(e) functor (straight from global
// memory); the last stage leaves its outputs in registers, register u R + r holding
// element j + r Ns (see p2_out_pos).  Between stages the values cross one shared buffer
// whose index is padded by one element per 16 (spad), which keeps the Stockham strides
// free of bank conflicts.  W transforms are interleaved column-wise in the buffer
// (element e of transform c at spad(e) W + c) so that W consecutive threads serve W
// consecutive columns of a row-major array.
#pragma once
#include "fft.cuh"

namespace dgt {

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n >> 1); }
__device__ __forceinline__ int spad(int e) { return e + (e >> 4); }

template <int N> struct Pow2 {
    static_assert(N >= 16 && N <= 16384 && (N & (N - 1)) == 0, "power of two in [16, 16384]");
    static constexpr int LOG = ilog2c(N);
    static constexpr int G = N / 16;
    static constexpr int NST = (LOG + 3) / 4;
    static constexpr int radix(int s) { return (s < NST - 1 || (LOG & 3) == 0) ? 16 : (1 << (LOG & 3)); }
    static constexpr int ns(int s) { return s == 0 ? 1 : ns(s - 1) * radix(s - 1); }
    static constexpr int RL = radix(NST - 1);          // last radix
    static constexpr int NSL = N / RL;                 // Ns of the last stage
    static constexpr int SMEM = N + N / 16;            // padded elements per transform
};

// element index held by register idx of thread t after the last stage
template <int N> __device__ __forceinline__ int p2_out_pos(int t, int idx) {
    using P = Pow2<N>;
    const int u = idx / P::RL, r = idx % P::RL;
    return t + P::G * u + r * P::NSL;
}

// FA: exchange addresses as one base per butterfly plus compile-time offsets (fewer integer
// instructions); !FA recomputes each padded index (fewer live registers, which the kernels
// that hold a second set of 16 values need to stay within 128)
template <int N, int DIR, int W, int S, bool FA, bool PK, typename C>
__device__ __forceinline__ void p2_stages(int c, int t, C* sm, const C* __restrict__ tw, C (&v)[16]) {
    using P = Pow2<N>;
    constexpr int Rp = P::radix(S - 1);
    constexpr int Nsp = P::ns(S - 1);
    constexpr int Bp = 16 / Rp;
    // padded positions: the writes of a butterfly are base + r Nsp with Rp = 16 (only the last
    // stage has a smaller radix, and it writes nothing); Nsp is 1 or a multiple of 16, so
    // spad(base + r Nsp) = spad(base) + r (Nsp + Nsp / 16) (for Nsp = 1, base is a multiple of
    // 16 and r < 16): one base address per butterfly plus compile-time offsets
    static_assert(Rp == 16, "only the last stage has a radix below 16");
    static_assert(Nsp == 1 || Nsp % 16 == 0, "Ns is a power of 16");
    constexpr int WSTEP = Nsp == 1 ? 1 : Nsp + Nsp / 16;
#pragma unroll
    for (int u = 0; u < Bp; ++u) {
        const int j = t + P::G * u;
        const int base = (j / Nsp) * Nsp * Rp + (j % Nsp);
        if constexpr (FA) {
            C* dst = sm + spad(base) * W + c;
#pragma unroll
            for (int r = 0; r < Rp; ++r) dst[r * WSTEP * W] = v[u * Rp + r];
        } else {
#pragma unroll
            for (int r = 0; r < Rp; ++r) sm[spad(base + r * Nsp) * W + c] = v[u * Rp + r];
        }
    }
    __syncthreads();
    constexpr int R = P::radix(S);
    constexpr int Ns = P::ns(S);
    constexpr int B = 16 / R;
    constexpr int NR = N / R;
    constexpr int TS = N / (Ns * R);
    // reads j + r NR, NR = N / R a multiple of 16: spad(j) + r (NR + NR / 16)
    static_assert(NR % 16 == 0, "stage stride a multiple of the padding period");
    constexpr int RSTEP = NR + NR / 16;
#pragma unroll
    for (int u = 0; u < B; ++u) {
        const int j = t + P::G * u;
        const int k = j % Ns;
        const C* src = sm + spad(j) * W + c;
        auto rd = [&](int r) -> C { return FA ? src[r * RSTEP * W] : sm[spad(j + r * NR) * W + c]; };
        if constexpr (sizeof(C) == 8) {
            // float: one first-order twiddle w = exp(DIR 2 pi i k / (Ns R)) per butterfly, from the
            // base table (stride 1) or the stage's compact table; w^r by a product tree of depth
            // ceil(log2 r) <= 4, i.e. a few float roundings, instead of R - 1 strided loads
            C wp[R];
            wp[1] = __ldg(tw + (TS == 1 ? k : N + Ns + k));
            if (DIR > 0) wp[1].y = -wp[1].y;
#pragma unroll
            for (int r = 2; r < R; ++r) wp[r] = cmul(wp[r / 2], wp[r - r / 2]);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const C x = rd(r);
                v[u * R + r] = r > 0 ? cmul(x, wp[r]) : x;
            }
        } else {
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C x = rd(r);
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
    for (int u = 0; u < B; ++u) dft_small<R, DIR, PK>(v + u * R);
    if constexpr (S + 1 < P::NST) p2_stages<N, DIR, W, S + 1, FA, PK>(c, t, sm, tw, v);
}

// Twiddle table of a length-N transform (built on the host): tw[e] = exp(-2 pi i e / N) for
// e < N, followed, for every stage S >= 1 with N / (Ns R) > 1 (so R = 16, Ns = 16^S), by the
// compact first-order twiddles tw[N + Ns + k] = exp(-2 pi i k / (16 Ns)), k < Ns.  The stage
// ranges [N + Ns, N + 2 Ns) are disjoint and end below 2 N.
// Full transform: v receives the outputs (positions from p2_out_pos).  All threads of the
// block must call it (it synchronises the block); `sm` holds Pow2<N>::SMEM * W elements.
template <int N, int DIR, int W, bool FA = true, bool PK = true, typename C, class Load>
__device__ __forceinline__ void fft_p2(int c, int t, C* sm, const C* __restrict__ tw, Load&& load, C (&v)[16]) {
    using P = Pow2<N>;
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = load(t + r * P::G);
    dft16<DIR, PK>(v);
    if constexpr (P::NST > 1) p2_stages<N, DIR, W, 1, FA, PK>(c, t, sm, tw, v);
}

// Register m of thread t holds element t + G m: the order stage 0 reads its inputs in.  The
// outputs of fft_p2 sit at the same positions in another order (p2_out_pos); output register
// idx holds element t + G p2_out_m(idx).  So the outputs of one transform can feed the next
// (of the same length) without leaving the registers: v_in[p2_out_m(idx)] = v_out[idx].
template <int N> __host__ __device__ constexpr int p2_out_m(int idx) {
    return idx / Pow2<N>::RL + (16 / Pow2<N>::RL) * (idx % Pow2<N>::RL);
}

// Full transform of the 16 values already in registers (v[m] = element t + G m).
template <int N, int DIR, int W, bool FA = true, bool PK = true, typename C>
__device__ __forceinline__ void fft_p2_regs(int c, int t, C* sm, const C* __restrict__ tw, C (&v)[16]) {
    using P = Pow2<N>;
    dft16<DIR, PK>(v);
    if constexpr (P::NST > 1) p2_stages<N, DIR, W, 1, FA, PK>(c, t, sm, tw, v);
}

}  // namespace dgt
