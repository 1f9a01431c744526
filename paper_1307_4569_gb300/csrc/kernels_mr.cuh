// Hot-path kernels for mixed-radix FFT lengths (fft_mr): the channel FFT with the route's
// post-processing (fft_post) and its adjoint (pre_ifft), for the lengths listed in MR_SWITCH;
// the same arithmetic as the power-of-two row kernels of kernels_p2.cuh, with the transform
// of fft_mr.cuh and indices reduced modulo N by comparison instead of masks.
#pragma once
#include "fft_mr.cuh"
#include "kernels_p2.cuh"

namespace dgt {

// rows per CTA: about 256 threads
template <class F> struct MrRow {
    static constexpr int RPB = F::G >= 256 ? 1 : 256 / F::G;
    static constexpr int THREADS = RPB * F::G;
};

template <int N> __device__ __forceinline__ int wrapn(int x) { return x >= N ? x - N : x; }

template <typename T, class F, bool SH1>
__global__ void __launch_bounds__(MrRow<F>::THREADS) fft_post_mr(const cplx<T>* __restrict__ y, cplx<T>* __restrict__ c,
                                                                 SepGeom g, int64_t J, int64_t rows_total,
                                                                 const cplx<T>* __restrict__ tw, PostParams<cplx<T>> pp) {
    using C = cplx<T>;
    constexpr int N = F::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gi = threadIdx.x / F::G, t = threadIdx.x % F::G;
    C* sm = reinterpret_cast<C*>(smem_raw) + gi * F::SMEM;
    const int64_t row = (int64_t)blockIdx.x * MrRow<F>::RPB + gi;
    const bool ok = row < rows_total;
    const C* yr = y + row * N;
    const int64_t b = ok ? (int64_t)pp.mJN.div((uint64_t)row) : 0;
    const int64_t rem = row - b * (int64_t)pp.mJN.d;
    const int64_t j = ok ? (int64_t)pp.mNs.div((uint64_t)rem) : 0, nn = ok ? rem - j * (int64_t)pp.mNs.d : 0;
    C v[F::V];
    if constexpr (SH1) {
        fft_mr<F, -1, 1>(0, t, sm, tw, [&](int k) -> C { return ok ? yr[k] : mk((T)0, (T)0); }, v);
        if (!ok) return;
        if (pp.sh1_fast) {
            const Sh1Row sr = sh1_row(pp, b, nn);
#pragma unroll
            for (int i = 0; i < F::OUT; ++i) {
                if (!mr_out_ok<F>(t, i)) continue;
                C ph;
                const int64_t o = sh1_at(pp, sr, mr_out_pos<F>(t, i), ph);
                c[o] = cmul(v[i], ph);
            }
            return;
        }
#pragma unroll
        for (int i = 0; i < F::OUT; ++i) {
            if (!mr_out_ok<F>(t, i)) continue;
            C ph;
            const int64_t o = out_index(pp, g, b, j, nn, mr_out_pos<F>(t, i), ph);
            c[o] = cmul(v[i], ph);
        }
    } else {
        RowMap<C> rm{};
        if (ok) rm = row_map(pp, g, b, j, nn);
        fft_mr<F, -1, 1>(0, t, sm, tw, [&](int k) -> C { return ok ? yr[k] : mk((T)0, (T)0); }, v);
        if (!ok) return;
        const int rot = (int)rm.rot;
        C* cb = c + rm.base;
#pragma unroll
        for (int i = 0; i < F::OUT; ++i)
            if (mr_out_ok<F>(t, i)) cb[wrapn<N>(mr_out_pos<F>(t, i) + rot)] = cmul(v[i], rm.ph);
    }
}

template <typename T, class F, bool SH1>
__global__ void __launch_bounds__(MrRow<F>::THREADS) pre_ifft_mr(const cplx<T>* __restrict__ c, cplx<T>* __restrict__ y,
                                                                 SepGeom g, int64_t J, int64_t rows_total,
                                                                 const cplx<T>* __restrict__ tw, PostParams<cplx<T>> pp) {
    using C = cplx<T>;
    constexpr int N = F::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gi = threadIdx.x / F::G, t = threadIdx.x % F::G;
    C* sm = reinterpret_cast<C*>(smem_raw) + gi * F::SMEM;
    const int64_t row = (int64_t)blockIdx.x * MrRow<F>::RPB + gi;
    const bool ok = row < rows_total;
    const int64_t b = ok ? (int64_t)pp.mJN.div((uint64_t)row) : 0;
    const int64_t rem = row - b * (int64_t)pp.mJN.d;
    const int64_t j = ok ? (int64_t)pp.mNs.div((uint64_t)rem) : 0, nn = ok ? rem - j * (int64_t)pp.mNs.d : 0;
    C v[F::V];
    if constexpr (SH1) {
        if (pp.sh1_fast) {
            const Sh1Row sr = sh1_row(pp, b, nn);
            fft_mr<F, +1, 1>(0, t, sm, tw, [&](int m) -> C {
                if (!ok) return mk((T)0, (T)0);
                C ph;
                const int64_t o = sh1_at(pp, sr, m, ph);
                return cmulc(c[o], ph);
            }, v);
        } else {
            fft_mr<F, +1, 1>(0, t, sm, tw, [&](int m) -> C {
                if (!ok) return mk((T)0, (T)0);
                C ph;
                const int64_t o = out_index(pp, g, b, j, nn, m, ph);
                return cmulc(c[o], ph);
            }, v);
        }
    } else {
        RowMap<C> rm{};
        if (ok) rm = row_map(pp, g, b, j, nn);
        const int rot = (int)rm.rot;
        const C* cb = c + (ok ? rm.base : 0);
        fft_mr<F, +1, 1>(0, t, sm, tw, [&](int m) -> C {
            return ok ? cmulc(cb[wrapn<N>(m + rot)], rm.ph) : mk((T)0, (T)0);
        }, v);
    }
    if (!ok) return;
    C* yr = y + row * N;
#pragma unroll
    for (int i = 0; i < F::OUT; ++i)
        if (mr_out_ok<F>(t, i)) yr[mr_out_pos<F>(t, i)] = v[i];
}

// ------------------------------------------------------------------------------------
// Frequency-shear rows in tiles.  When s1 = 0 and b is a multiple of C6, the output channel
// of Algorithm 1's reindex, kt = (C6 n mod L) / b = n / q with q = b / C6, depends on the row n
// alone, q rows make up one channel and N = q Nr.  A CTA then takes RT = q W consecutive rows of
// one signal, i.e. W whole output channels kt0 .. kt0 + W - 1.
//   fft_post_mr_tile: the rows' outputs, times their phases, go to shared memory by
//   destination (stage[mt W + kt - kt0]) and leave as runs of W channels per output time:
//   whole 32-byte sectors instead of one sector per 8-byte store.
//   pre_ifft_mr_tile: the W channels are read the same way, and each transform gathers its
//   inputs (times the conjugate phases) from shared memory.
// Same values as fft_post_mr / pre_ifft_mr with SH1 (sh1_split is sh1_at's map).
// ------------------------------------------------------------------------------------
// the two-level table of exp(2 pi i e / 2N) (pp.cis2N: hi[e >> shift], lo[e mod 2^shift]) copied
// into shared memory, so that the per-coefficient phase of the map is two shared loads; entries
// rounded up to an even count, which keeps what follows 16-byte aligned
template <typename C> struct SharedCis {
    const C* hi;
    const C* lo;
    int shift;
    __device__ __forceinline__ C at(uint32_t e) const { return cmul(hi[e >> shift], lo[e & ((1u << shift) - 1u)]); }
};
template <typename C> __host__ __device__ __forceinline__ uint32_t shared_cis_entries(const CisTable<C>& t) {
    const uint32_t nhi = (uint32_t)(t.md.d >> t.shift) + 1u;
    return (nhi + (1u << t.shift) + 1u) & ~1u;
}
template <typename C> __device__ __forceinline__ SharedCis<C> load_shared_cis(const CisTable<C>& t, C* buf) {
    const uint32_t nhi = (uint32_t)(t.md.d >> t.shift) + 1u, nlo = 1u << t.shift;
    for (uint32_t i = threadIdx.x; i < nhi; i += blockDim.x) buf[i] = t.hi[i];
    for (uint32_t i = threadIdx.x; i < nlo; i += blockDim.x) buf[nhi + i] = t.lo[i];
    return SharedCis<C>{buf, buf + nhi, t.shift};
}

template <typename T, class F, int W>
__global__ void __launch_bounds__(1024) fft_post_mr_tile(const cplx<T>* __restrict__ y, cplx<T>* __restrict__ c,
                                                         int64_t rows_per_signal, int q,
                                                         const cplx<T>* __restrict__ tw, PostParams<cplx<T>> pp) {
    using C = cplx<T>;
    constexpr int NR = F::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RT = q * W;
    const int gi = threadIdx.x / F::G, t = threadIdx.x % F::G;
    C* tab = reinterpret_cast<C*>(smem_raw);
    const SharedCis<C> cis = load_shared_cis(pp.cis2N, tab);
    C* stage = tab + shared_cis_entries(pp.cis2N);
    C* sm = stage + gi * F::SMEM;
    __syncthreads();
    const int64_t tiles = rows_per_signal / RT;
    const int64_t b = blockIdx.x / tiles;
    const int64_t n0 = (blockIdx.x - b * tiles) * RT;
    const int64_t nn = n0 + gi;
    const uint32_t kt0 = (uint32_t)(n0 / q);
    const int jj = gi / q;                         // this row's channel, kt - kt0
    const C* yr = y + (b * rows_per_signal + nn) * NR;
    const Sh1Row sr = sh1_row(pp, b, nn);
    C v[F::V];
    fft_mr<F, -1, 1>(0, t, sm, tw, [&](int k) -> C { return yr[k]; }, v);
    // the transforms' last exchange reads came before their final barrier: the buffer is free
#pragma unroll
    for (int i = 0; i < F::OUT; ++i) {
        if (!mr_out_ok<F>(t, i)) continue;
        uint32_t e, mt;
        sh1_index_t(pp, sr, mr_out_pos<F>(t, i), e, mt);
        stage[mt * W + jj] = cmul(v[i], cis.at(e));
    }
    __syncthreads();
    C* cb = c + sr.base + kt0;
    const int total = (int)pp.f_N * W;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x)
        cb[(int64_t)(idx / W) * pp.M + idx % W] = stage[idx];
}

template <typename T, class F, int W>
__global__ void __launch_bounds__(1024) pre_ifft_mr_tile(const cplx<T>* __restrict__ c, cplx<T>* __restrict__ y,
                                                         int64_t rows_per_signal, int q,
                                                         const cplx<T>* __restrict__ tw, PostParams<cplx<T>> pp) {
    using C = cplx<T>;
    constexpr int NR = F::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int RT = q * W;
    const int gi = threadIdx.x / F::G, t = threadIdx.x % F::G;
    C* tab = reinterpret_cast<C*>(smem_raw);
    const SharedCis<C> cis = load_shared_cis(pp.cis2N, tab);
    C* stage = tab + shared_cis_entries(pp.cis2N);
    C* sm = stage + (size_t)pp.f_N * W + gi * F::SMEM;
    const int64_t tiles = rows_per_signal / RT;
    const int64_t b = blockIdx.x / tiles;
    const int64_t n0 = (blockIdx.x - b * tiles) * RT;
    const int64_t nn = n0 + gi;
    const uint32_t kt0 = (uint32_t)(n0 / q);
    const int jj = gi / q;                         // this row's channel, kt - kt0
    const Sh1Row sr = sh1_row(pp, b, nn);
    const C* cb = c + sr.base + kt0;
    const int total = (int)pp.f_N * W;
    // the tile, eight loads in flight per thread
    constexpr int U = 8;
    for (int i0 = threadIdx.x; i0 < total; i0 += U * (int)blockDim.x) {
        C x[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int idx = i0 + u * (int)blockDim.x;
            x[u] = idx < total ? cb[(int64_t)(idx / W) * pp.M + idx % W] : mk((T)0, (T)0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (i0 + u * (int)blockDim.x < total) stage[i0 + u * (int)blockDim.x] = x[u];
    }
    __syncthreads();
    C v[F::V];
    fft_mr<F, +1, 1>(0, t, sm, tw, [&](int m) -> C {
        uint32_t e, mt;
        sh1_index_t(pp, sr, m, e, mt);
        return cmulc(stage[mt * W + jj], cis.at(e));
    }, v);
    C* yr = y + (b * rows_per_signal + nn) * NR;
#pragma unroll
    for (int i = 0; i < F::OUT; ++i)
        if (mr_out_ok<F>(t, i)) yr[mr_out_pos<F>(t, i)] = v[i];
}

// ------------------------------------------------------------------------------------
// column kernels (transforms along the strided dimension, W adjacent columns per CTA): the
// Zak transform, the block product with the inverse FFT over xi, its adjoint, and the inverse
// Zak transform -- the arithmetic of zak_fwd_p2, prod_ifft_p2, fft_prod_adj_p2, zak_inv_p2
// ------------------------------------------------------------------------------------
template <typename T, class F> struct MrCol {
    static constexpr int WMAX = sizeof(T) == 4 ? 8 : 4;
    static constexpr int WT = 512 / F::G < 1 ? 1 : 512 / F::G;
    static constexpr int W = WMAX < WT ? WMAX : WT;
    static constexpr int THREADS = W * F::G;
    static constexpr size_t SMEM = sizeof(cplx<T>) * (size_t)F::SMEM * W;
    // the adjoint holds its accumulators beside the transform: at most 128 registers a thread
    static constexpr int MINB_ADJ = 65536 / (THREADS * 128) > 0 ? 65536 / (THREADS * 128) : 1;
};

template <typename T, class F>
__global__ void __launch_bounds__(MrCol<T, F>::THREADS) zak_fwd_mr(const void* __restrict__ src, int src_real,
                                                                   int64_t sbs, cplx<T>* __restrict__ zf, int64_t zbs,
                                                                   int64_t K0, const cplx<T>* __restrict__ tw,
                                                                   ChirpParams<cplx<T>> pre) {
    using C = cplx<T>;
    using CF = MrCol<T, F>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.y;
    const int64_t col = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = col < K0;
    C v[F::V];
    fft_mr<F, -1, CF::W>(c, t, sm, tw, [&](int e) -> C {
        if (!ok) return mk((T)0, (T)0);
        const int64_t l = col + K0 * e;
        C x = load_any<C>(src, src_real, b * sbs + l);
        if (pre.mode == PRE_CHIRP) x = cmul(x, chirp_factor(pre, l));
        return x;
    }, v);
    if (!ok) return;
#pragma unroll
    for (int i = 0; i < F::OUT; ++i)
        if (mr_out_ok<F>(t, i)) zf[b * zbs + (int64_t)mr_out_pos<F>(t, i) * K0 + col] = v[i];
}

template <typename T, class F>
__global__ void __launch_bounds__(MrCol<T, F>::THREADS) prod_ifft_mr(const cplx<T>* __restrict__ zf,
                                                                     const cplx<T>* __restrict__ zg,
                                                                     cplx<T>* __restrict__ y, SepGeom g, int64_t J,
                                                                     const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using CF = MrCol<T, F>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.z;
    const int64_t j = (int)blockIdx.y / (int)g.q, w = (int)blockIdx.y % (int)g.q;
    const int64_t k = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = k < g.M;
    int64_t colG = k - g.a * w;
    const bool wrap = colG < 0;
    if (wrap) colG += g.K0;
    const C* zfb = zf + b * g.L + k;
    const C* zgj = zg + j * g.L + colG;
    C v[F::V];
    fft_mr<F, +1, CF::W>(c, t, sm, tw, [&](int xi) -> C {
        if (!ok) return mk((T)0, (T)0);
        C x = cmulc(zfb[(int64_t)xi * g.K0], zgj[(int64_t)xi * g.K0]);
        if (wrap) x = cmulc(x, __ldg(tw + xi));
        return x;
    }, v);
    if (!ok) return;
    const T scale = (T)1 / (T)F::N;
    C* yb = y + ((b * J + j) * g.d * g.q + w) * g.M + k;
#pragma unroll
    for (int i = 0; i < F::OUT; ++i)
        if (mr_out_ok<F>(t, i)) yb[(int64_t)g.q * mr_out_pos<F>(t, i) * g.M] = cscale(v[i], scale);
}

template <typename T, class F>
__global__ void __launch_bounds__(MrCol<T, F>::THREADS, MrCol<T, F>::MINB_ADJ) fft_prod_adj_mr(const cplx<T>* __restrict__ y,
                                                                        const cplx<T>* __restrict__ zg,
                                                                        cplx<T>* __restrict__ zf, SepGeom g, int64_t J,
                                                                        const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using CF = MrCol<T, F>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = k < g.M;
    const T scale = (T)1 / (T)F::N;
    C acc[F::OUT];
#pragma unroll
    for (int i = 0; i < F::OUT; ++i) acc[i] = mk((T)0, (T)0);
    for (int64_t j = 0; j < J; ++j) {
        for (int64_t w = 0; w < g.q; ++w) {
            const C* yb = y + ((b * J + j) * g.d * g.q + w) * g.M + k;
            C v[F::V];
            fft_mr<F, -1, CF::W>(c, t, sm, tw, [&](int nu) -> C {
                return ok ? yb[(int64_t)g.q * nu * g.M] : mk((T)0, (T)0);
            }, v);
            int64_t colG = k - g.a * w;
            const bool wrap = colG < 0;
            if (wrap) colG += g.K0;
            const C* zgj = zg + j * g.L + colG;
            if (ok) {
#pragma unroll
                for (int i = 0; i < F::OUT; ++i) {
                    if (!mr_out_ok<F>(t, i)) continue;
                    const int xi = mr_out_pos<F>(t, i);
                    C u = cmul(cscale(v[i], scale), zgj[(int64_t)xi * g.K0]);
                    if (wrap) u = cmul(u, __ldg(tw + xi));
                    acc[i] = cadd(acc[i], u);
                }
            }
            __syncthreads();          // the next transform reuses the exchange buffer
        }
    }
    if (!ok) return;
#pragma unroll
    for (int i = 0; i < F::OUT; ++i)
        if (mr_out_ok<F>(t, i)) zf[b * g.L + (int64_t)mr_out_pos<F>(t, i) * g.K0 + k] = acc[i];
}

template <typename T, class F>
__global__ void __launch_bounds__(MrCol<T, F>::THREADS) zak_inv_mr(const cplx<T>* __restrict__ zf, int64_t zbs,
                                                                   void* __restrict__ dst, int dst_real, int64_t dbs,
                                                                   int64_t K0, const cplx<T>* __restrict__ tw,
                                                                   ChirpParams<cplx<T>> post, T scale) {
    using C = cplx<T>;
    using CF = MrCol<T, F>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.y;
    const int64_t col = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = col < K0;
    C v[F::V];
    fft_mr<F, +1, CF::W>(c, t, sm, tw, [&](int xi) -> C {
        return ok ? zf[b * zbs + (int64_t)xi * K0 + col] : mk((T)0, (T)0);
    }, v);
    if (!ok) return;
#pragma unroll
    for (int i = 0; i < F::OUT; ++i) {
        if (!mr_out_ok<F>(t, i)) continue;
        const int64_t l = col + K0 * mr_out_pos<F>(t, i);
        C x = cscale(v[i], scale);
        if (post.mode == PRE_CHIRP) x = cmul(x, chirp_factor(post, l));
        store_any(dst, dst_real, b * dbs + l, x);
    }
}

// ------------------------------------------------------------------------------------
// The length-L transform of the frequency-shear branch as four steps, L = L1 L2, with compiled
// transforms of both factors (the arithmetic of fftL_cols_kernel / fftL_rows_kernel):
//   cols: DFT over n1 of x[n1 L2 + n2] (pre-chirp on load), times exp(dir 2 pi i n2 k1 / L),
//         into tmp[k1 L2 + n2]; W columns n2 per CTA.  n2 k1 < L needs no reduction.
//   rows: DFT over n2 of tmp[k1 L2 + .] per row k1, into dst[k1 + L1 k2] scaled and
//         post-chirped; the rows of a CTA go through shared memory so that the transposed
//         store writes runs of consecutive k1.
// ------------------------------------------------------------------------------------
template <typename T, class F, int DIR>
__global__ void __launch_bounds__(MrCol<T, F>::THREADS) fftL_cols_mr(const void* __restrict__ src, int src_real,
                                                                     cplx<T>* __restrict__ tmp, int64_t L2,
                                                                     const cplx<T>* __restrict__ tw,
                                                                     ChirpParams<cplx<T>> pre, CisTable<cplx<T>> cisL) {
    using C = cplx<T>;
    using CF = MrCol<T, F>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.y;
    const int64_t L = (int64_t)F::N * L2;
    const int64_t col = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = col < L2;
    C v[F::V];
    fft_mr<F, DIR, CF::W>(c, t, sm, tw, [&](int e) -> C {
        if (!ok) return mk((T)0, (T)0);
        const int64_t l = col + L2 * e;
        C x = load_any<C>(src, src_real, b * L + l);
        if (pre.mode == PRE_CHIRP) x = cmul(x, chirp_factor(pre, l));
        return x;
    }, v);
    if (!ok) return;
#pragma unroll
    for (int i = 0; i < F::OUT; ++i) {
        if (!mr_out_ok<F>(t, i)) continue;
        const int64_t k1 = mr_out_pos<F>(t, i);
        const uint64_t ex = (uint64_t)(col * k1);
        const C w = cisL.at(DIR < 0 ? (ex ? (uint64_t)L - ex : 0) : ex);
        tmp[b * L + k1 * L2 + col] = cmul(v[i], w);
    }
}

template <typename T, class F, int DIR>
__global__ void __launch_bounds__(MrRow<F>::THREADS) fftL_rows_mr(const cplx<T>* __restrict__ tmp, void* __restrict__ dst,
                                                                  int dst_real, int64_t L1,
                                                                  const cplx<T>* __restrict__ tw,
                                                                  ChirpParams<cplx<T>> post, T scale) {
    using C = cplx<T>;
    using RC = MrRow<F>;
    constexpr int L2 = F::N;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gi = threadIdx.x / F::G, t = threadIdx.x % F::G;
    C* sm = reinterpret_cast<C*>(smem_raw) + gi * F::SMEM;
    C* stage = reinterpret_cast<C*>(smem_raw);                 // [k2][RPB] after the transforms
    const int64_t b = blockIdx.y;
    const int64_t L = L1 * L2;
    const int64_t r0 = (int64_t)blockIdx.x * RC::RPB;
    const int64_t r = r0 + gi;
    const bool ok = r < L1;
    C v[F::V];
    fft_mr<F, DIR, 1>(0, t, sm, tw, [&](int k) -> C { return ok ? tmp[b * L + r * L2 + k] : mk((T)0, (T)0); }, v);
    // the transforms' last exchange reads came before their final barrier: the buffer is free
#pragma unroll
    for (int i = 0; i < F::OUT; ++i)
        if (mr_out_ok<F>(t, i)) stage[mr_out_pos<F>(t, i) * RC::RPB + gi] = v[i];
    __syncthreads();
    const int nr = (int)min((int64_t)RC::RPB, L1 - r0);
    for (int idx = threadIdx.x; idx < L2 * RC::RPB; idx += RC::THREADS) {
        const int k2 = idx / RC::RPB, rr = idx % RC::RPB;
        if (rr >= nr) continue;
        const int64_t kk = r0 + rr + L1 * (int64_t)k2;
        C x = cscale(stage[idx], scale);
        if (post.mode == PRE_CHIRP) x = cmul(x, chirp_factor(post, kk));
        store_any(dst, dst_real, b * L + kk, x);
    }
}

// ------------------------------------------------------------------------------------
// the lengths with a compiled mixed-radix transform: N, threads per transform, radices
// ------------------------------------------------------------------------------------
using Mr60 = Mixed<60, 4, RadixList<4, 15>>;
using Mr120 = Mixed<120, 8, RadixList<8, 15>>;
using Mr180 = Mixed<180, 12, RadixList<4, 5, 9>>;
using Mr240 = Mixed<240, 16, RadixList<16, 15>>;
using Mr360 = Mixed<360, 24, RadixList<8, 9, 5>>;
using Mr480 = Mixed<480, 32, RadixList<16, 2, 15>>;
using Mr720 = Mixed<720, 48, RadixList<16, 9, 5>>;
using Mr960 = Mixed<960, 64, RadixList<16, 4, 15>>;
using Mr2160 = Mixed<2160, 144, RadixList<16, 9, 15>>;

#define MR_SWITCH(NV, ...)                                \
    switch (NV) {                                          \
        case 60: { using FF = Mr60; __VA_ARGS__; }                \
        case 120: { using FF = Mr120; __VA_ARGS__; }              \
        case 180: { using FF = Mr180; __VA_ARGS__; }              \
        case 240: { using FF = Mr240; __VA_ARGS__; }              \
        case 360: { using FF = Mr360; __VA_ARGS__; }              \
        case 480: { using FF = Mr480; __VA_ARGS__; }              \
        case 720: { using FF = Mr720; __VA_ARGS__; }              \
        case 960: { using FF = Mr960; __VA_ARGS__; }              \
        case 2160: { using FF = Mr2160; __VA_ARGS__; }            \
        default: return cudaErrorNotSupported;             \
    }

template <typename T, class F, bool POST>
cudaError_t mr_rows_n(const cplx<T>* src, cplx<T>* dst, const SepGeom& g, int64_t J, const void* tw,
                      const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    if (pp.half) return cudaErrorNotSupported;
    using RC = MrRow<F>;
    const size_t smem = sizeof(cplx<T>) * (size_t)F::SMEM * RC::RPB;
    const bool sh1 = pp.mode == POST_SHEAR1;
    if (sh1 && pp.sh1_fast && pp.f_s1ar == 0 && J == 1 && pp.f_C6 > 0 && pp.qb.d % pp.f_C6 == 0) {
        // tiles of q W rows = W whole output channels (see fft_post_mr_tile): every condition
        // that keeps the tile's channels in [kt0, kt0 + W) and its stage inside shared memory
        constexpr int W = 2;
        const int64_t q = pp.qb.d / pp.f_C6;
        const int64_t rps = g.d * g.q;                 // rows per signal
        const int64_t RT = q * W;
        const size_t stage = sizeof(cplx<T>) * (size_t)pp.f_N * W;
        const size_t fsm = sizeof(cplx<T>) * (size_t)F::SMEM * (size_t)RT;
        const size_t tsm = sizeof(cplx<T>) * (size_t)shared_cis_entries(pp.cis2N) + (POST ? std::max(stage, fsm) : stage + fsm);
        if ((int64_t)pp.f_N == q * F::N && rps % RT == 0 && rps / q <= (int64_t)pp.f_M &&
            (uint64_t)pp.f_C6 * (uint64_t)(rps - 1) < (uint64_t)pp.qL.d && RT * F::G <= 1024 && tsm <= kSmemBudget) {
            auto kt = POST ? fft_post_mr_tile<T, F, W> : pre_ifft_mr_tile<T, F, W>;
            cudaError_t e = p2_smem(kt, tsm);
            if (e != cudaSuccess) return e;
            kt<<<(unsigned)(B * (rps / RT)), (unsigned)(RT * F::G), tsm, st>>>(src, dst, rps, (int)q,
                                                                           (const cplx<T>*)tw, pp);
            return cudaGetLastError();
        }
    }
    auto k = POST ? (sh1 ? fft_post_mr<T, F, true> : fft_post_mr<T, F, false>)
                  : (sh1 ? pre_ifft_mr<T, F, true> : pre_ifft_mr<T, F, false>);
    cudaError_t e = p2_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = B * J * g.d * g.q;
    PostParams<cplx<T>> q = pp;
    q.mJN = make_mod((uint64_t)(J * g.d * g.q));
    q.mNs = make_mod((uint64_t)(g.d * g.q));
    k<<<(unsigned)((rows + RC::RPB - 1) / RC::RPB), RC::THREADS, smem, st>>>(src, dst, g, J, rows,
                                                                            (const cplx<T>*)tw, q);
    return cudaGetLastError();
}

// run-time dispatch; cudaErrorNotSupported = a length without a compiled transform
template <typename T>
cudaError_t mr_fft_post(const cplx<T>* y, cplx<T>* c, const SepGeom& g, int64_t J, const void* tw,
                        const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    MR_SWITCH(g.M, return (mr_rows_n<T, FF, true>(y, c, g, J, tw, pp, B, st)))
}
template <typename T>
cudaError_t mr_pre_ifft(const cplx<T>* c, cplx<T>* y, const SepGeom& g, int64_t J, const void* tw,
                        const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    MR_SWITCH(g.M, return (mr_rows_n<T, FF, false>(c, y, g, J, tw, pp, B, st)))
}

// column launchers; cudaErrorNotSupported = a length without a compiled transform (or p != 1)
template <typename T, class F, class K> cudaError_t mr_col_prep(K k) { return p2_smem(k, MrCol<T, F>::SMEM); }

template <typename T>
cudaError_t mr_zak_fwd(const void* src, int src_real, int64_t sbs, cplx<T>* zf, int64_t zbs, int64_t d, int64_t K0,
                       const void* tw, const ChirpParams<cplx<T>>& pre, int64_t B, cudaStream_t st) {
    MR_SWITCH(d, {
        using CF = MrCol<T, FF>;
        auto k = zak_fwd_mr<T, FF>;
        cudaError_t e = mr_col_prep<T, FF>(k);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((K0 + CF::W - 1) / CF::W), (unsigned)B);
        k<<<grid, CF::THREADS, CF::SMEM, st>>>(src, src_real, sbs, zf, zbs, K0, (const cplx<T>*)tw, pre);
        return cudaGetLastError();
    })
}
template <typename T>
cudaError_t mr_prod_ifft(const cplx<T>* zf, const cplx<T>* zg, int64_t J, cplx<T>* y, const SepGeom& g,
                         const void* tw, int64_t B, cudaStream_t st) {
    if (g.p != 1) return cudaErrorNotSupported;
    MR_SWITCH(g.d, {
        using CF = MrCol<T, FF>;
        auto k = prod_ifft_mr<T, FF>;
        cudaError_t e = mr_col_prep<T, FF>(k);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((g.M + CF::W - 1) / CF::W), (unsigned)(J * g.q), (unsigned)B);
        k<<<grid, CF::THREADS, CF::SMEM, st>>>(zf, zg, y, g, J, (const cplx<T>*)tw);
        return cudaGetLastError();
    })
}
template <typename T>
cudaError_t mr_fft_prod_adj(const cplx<T>* y, const cplx<T>* zg, int64_t J, cplx<T>* zf, const SepGeom& g,
                            const void* tw, int64_t B, cudaStream_t st) {
    if (g.p != 1) return cudaErrorNotSupported;
    MR_SWITCH(g.d, {
        using CF = MrCol<T, FF>;
        auto k = fft_prod_adj_mr<T, FF>;
        cudaError_t e = mr_col_prep<T, FF>(k);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((g.M + CF::W - 1) / CF::W), (unsigned)B);
        k<<<grid, CF::THREADS, CF::SMEM, st>>>(y, zg, zf, g, J, (const cplx<T>*)tw);
        return cudaGetLastError();
    })
}
template <typename T>
cudaError_t mr_zak_inv(const cplx<T>* zf, int64_t zbs, void* dst, int dst_real, int64_t dbs, int64_t d, int64_t K0,
                       const void* tw, const ChirpParams<cplx<T>>& post, T scale, int64_t B, cudaStream_t st) {
    MR_SWITCH(d, {
        using CF = MrCol<T, FF>;
        auto k = zak_inv_mr<T, FF>;
        cudaError_t e = mr_col_prep<T, FF>(k);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((K0 + CF::W - 1) / CF::W), (unsigned)B);
        k<<<grid, CF::THREADS, CF::SMEM, st>>>(zf, zbs, dst, dst_real, dbs, K0, (const cplx<T>*)tw, post, scale);
        return cudaGetLastError();
    })
}

template <typename T>
cudaError_t mr_fftL_cols(const void* src, int src_real, cplx<T>* tmp, int64_t L1, int64_t L2, int dir, const void* tw,
                         const ChirpParams<cplx<T>>& pre, const CisTable<cplx<T>>& cisL, int64_t B, cudaStream_t st) {
    MR_SWITCH(L1, {
        using CF = MrCol<T, FF>;
        auto k = dir < 0 ? fftL_cols_mr<T, FF, -1> : fftL_cols_mr<T, FF, +1>;
        cudaError_t e = mr_col_prep<T, FF>(k);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((L2 + CF::W - 1) / CF::W), (unsigned)B);
        k<<<grid, CF::THREADS, CF::SMEM, st>>>(src, src_real, tmp, L2, (const cplx<T>*)tw, pre, cisL);
        return cudaGetLastError();
    })
}
template <typename T>
cudaError_t mr_fftL_rows(const cplx<T>* tmp, void* dst, int dst_real, int64_t L1, int64_t L2, int dir, const void* tw,
                         const ChirpParams<cplx<T>>& post, T scale, int64_t B, cudaStream_t st) {
    MR_SWITCH(L2, {
        using RC = MrRow<FF>;
        auto k = dir < 0 ? fftL_rows_mr<T, FF, -1> : fftL_rows_mr<T, FF, +1>;
        const size_t smem = sizeof(cplx<T>) * (size_t)FF::SMEM * RC::RPB;
        cudaError_t e = p2_smem(k, smem);
        if (e != cudaSuccess) return e;
        dim3 grid((unsigned)((L1 + RC::RPB - 1) / RC::RPB), (unsigned)B);
        k<<<grid, RC::THREADS, smem, st>>>(tmp, dst, dst_real, L1, (const cplx<T>*)tw, post, scale);
        return cudaGetLastError();
    })
}

}  // namespace dgt
