// Hot-path kernels for power-of-two FFT lengths (fft_p2).  Same arithmetic as the generic
// kernels of engine_zak.cu / engine_aux.cu (see their comments for the formulas), with the
// first FFT stage fused into the global loads and the last into the global stores.
//
// Column kernels transform along the strided dimension of a row-major [n][cols] array:
// W consecutive columns share a CTA (W * N/16 threads), so every load and store instruction
// touches W consecutive elements of a row.  Row kernels transform contiguous rows: RPB rows
// per CTA, N/16 threads each.
#pragma once
#include <type_traits>

#include "fft_p2.cuh"
#include "kcommon.cuh"
#include "tma.cuh"

namespace dgt {

template <typename T, int N> struct ColCfg {
    static constexpr int G = N / 16;
    static constexpr int WMAX = sizeof(T) == 4 ? 8 : 4;
    static constexpr int WT = (512 / G) < 1 ? 1 : (512 / G);                           // <= 512 threads
    static constexpr int WS = (int)(kSmemBudget / (sizeof(cplx<T>) * (size_t)Pow2<N>::SMEM));
    static constexpr int W = WMAX < WT ? (WMAX < WS ? WMAX : WS) : (WT < WS ? WT : WS);  // columns per CTA
    static constexpr int THREADS = W * G;
    static constexpr size_t SMEM = sizeof(cplx<T>) * (size_t)Pow2<N>::SMEM * W;
    // blocks per SM the register allocation must allow: 64 registers a thread in float32,
    // 128 in float64 (the 16 complex values of a thread take 32 / 64 of them)
    static constexpr int MINB = (sizeof(T) == 4 ? 2048 : 1024) / (THREADS * 2) > 0
                                    ? (sizeof(T) == 4 ? 2048 : 1024) / (THREADS * 2) : 1;
    static_assert(W >= 1, "tile does not fit");
};

// fft_prod_adj (two sets of 16 values per thread, the transform and the accumulators): float
// tiles of half the columns, two CTAs per SM (<= 128 registers), so that one CTA computes while
// the other waits at an exchange barrier (2.32 -> 2.16 ms on 64 audio signals; zak_prod_ifft,
// which holds its Zak column the same way, got slower with it and keeps the full tiles)
template <typename T, int N> struct AdjCfg {
    using Base = ColCfg<T, N>;
    static constexpr bool HALVE = sizeof(T) == 4 && N >= 1024 && Base::W >= 2;
    static constexpr int W = HALVE ? Base::W / 2 : Base::W;
    static constexpr int THREADS = W * Base::G;
    static constexpr size_t SMEM = sizeof(cplx<T>) * (size_t)Pow2<N>::SMEM * W;
    static constexpr int MINB = HALVE ? 2 : 1;
};

// FIR analysis: CTAs of 128 threads (two rows for M = 1024), so that a dozen CTAs of 64-register
// threads share an SM and the staging of one overlaps the transforms of the others (1.87 -> 1.73
// ms against 256-thread CTAs on 64 audio signals)
template <int N> struct AnaCfg {
    static constexpr int G = N / 16;
    static constexpr int RPB = G >= 128 ? 1 : 128 / G;
    static constexpr int THREADS = RPB * G;
    static constexpr int MINB = 65536 / (THREADS * 64) > 0 ? 65536 / (THREADS * 64) : 1;
};

template <int N> struct RowCfg {
    static constexpr int G = N / 16;
    static constexpr int RPB = G >= 256 ? 1 : 256 / G;                   // rows per CTA
    static constexpr int THREADS = RPB * G;
    static constexpr int MINB = 65536 / (THREADS * 64) > 0 ? 65536 / (THREADS * 64) : 1;   // <= 64 registers
};

template <typename K> static cudaError_t p2_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

// ------------------------------------------------------------------------------------
// zak_fwd: ZF[b][xi][col] = sum_mu x(col + K0 mu) e^{-2 pi i mu xi / d}   (d = N)
// ------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(ColCfg<T, N>::THREADS) zak_fwd_p2(const void* __restrict__ src, int src_real,
                                                                    int64_t sbs, cplx<T>* __restrict__ zf,
                                                                    int64_t zbs, int64_t K0,
                                                                    const cplx<T>* __restrict__ tw,
                                                                    ChirpParams<cplx<T>> pre) {
    using C = cplx<T>;
    using CF = ColCfg<T, N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.y;
    const int64_t col = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = col < K0;
    C v[16];
    fft_p2<N, -1, CF::W>(c, t, sm, tw, [&](int e) -> C {
        if (!ok) return mk((T)0, (T)0);
        const int64_t l = col + K0 * e;
        C x = load_any<C>(src, src_real, b * sbs + l);
        if (pre.mode == PRE_CHIRP) x = cmul(x, chirp_factor(pre, l));
        return x;
    }, v);
    if (ok) {
#pragma unroll
        for (int i = 0; i < 16; ++i) zf[b * zbs + (int64_t)p2_out_pos<N>(t, i) * K0 + col] = v[i];
    }
}

// ------------------------------------------------------------------------------------
// prod_ifft (p = 1): X_w[xi][k] = ZF[xi][k] conj(ZG~_j[xi][k - a w]), inverse FFT over xi,
// Y[b][j][w + q nu][k] = h / d.   grid (k-blocks, J q, B)
// ------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(ColCfg<T, N>::THREADS, ColCfg<T, N>::MINB) prod_ifft_p2(const cplx<T>* __restrict__ zf,
                                                                      const cplx<T>* __restrict__ zg,
                                                                      cplx<T>* __restrict__ y, SepGeom g, int64_t J,
                                                                      const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using CF = ColCfg<T, N>;
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
    C v[16];
    fft_p2<N, +1, CF::W>(c, t, sm, tw, [&](int xi) -> C {
        if (!ok) return mk((T)0, (T)0);
        C x = cmulc(zfb[(int64_t)xi * g.K0], zgj[(int64_t)xi * g.K0]);
        if (wrap) x = cmulc(x, __ldg(tw + xi));
        return x;
    }, v);
    if (ok) {
        const T scale = (T)1 / (T)N;
        C* yb = y + ((b * J + j) * g.d * g.q + w) * g.M + k;
#pragma unroll
        for (int i = 0; i < 16; ++i) yb[(int64_t)g.q * p2_out_pos<N>(t, i) * g.M] = cscale(v[i], scale);
    }
}

// ------------------------------------------------------------------------------------
// fft_prod_adj (p = 1): for every (j, w) FFT over nu of Y'[b][j][w + q nu][k], / d, times
// ZG~_j[xi][k - a w], summed into ZF'[b][xi][k].   grid (k-blocks, B)
// ------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(AdjCfg<T, N>::THREADS, AdjCfg<T, N>::MINB) fft_prod_adj_p2(const cplx<T>* __restrict__ y,
                                                                         const cplx<T>* __restrict__ zg,
                                                                         cplx<T>* __restrict__ zf, SepGeom g,
                                                                         int64_t J, const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using CF = AdjCfg<T, N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = k < g.M;
    const T scale = (T)1 / (T)N;
    C acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = mk((T)0, (T)0);
    for (int64_t j = 0; j < J; ++j) {
        for (int64_t w = 0; w < g.q; ++w) {
            const C* yb = y + ((b * J + j) * g.d * g.q + w) * g.M + k;
            C v[16];
            fft_p2<N, -1, CF::W, false>(c, t, sm, tw, [&](int nu) -> C {
                return ok ? yb[(int64_t)g.q * nu * g.M] : mk((T)0, (T)0);
            }, v);
            int64_t colG = k - g.a * w;
            const bool wrap = colG < 0;
            if (wrap) colG += g.K0;
            const C* zgj = zg + j * g.L + colG;
            if (ok) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int xi = p2_out_pos<N>(t, i);
                    C u = cmul(cscale(v[i], scale), zgj[(int64_t)xi * g.K0]);
                    if (wrap) u = cmul(u, __ldg(tw + xi));
                    acc[i] = cadd(acc[i], u);
                }
            }
            __syncthreads();          // the next transform reuses the exchange buffer
        }
    }
    if (ok) {
#pragma unroll
        for (int i = 0; i < 16; ++i) zf[b * g.L + (int64_t)p2_out_pos<N>(t, i) * g.K0 + k] = acc[i];
    }
}

// ------------------------------------------------------------------------------------
// fft_prod_adj, float, with the column tiles of Y staged by the tensor memory accelerator:
// one thread issues the tile of the next (j, w) (d rows of W columns, in boxes of up to 256
// rows) into the other of two shared buffers while the CTA transforms the current one, so the
// transforms read shared memory instead of waiting on strided global loads.  ZGT: the window
// factor tile ZG~_j[.][k0 - a w ..] of the current (j, w) is copied the same way into the
// buffer whose Y values have just been read, during the transform; the Y tile two iterations
// ahead follows once the products are summed.  Waits are bounded
// (wait_limit cycles; 0 lets every wait expire at once, for tests); a CTA whose wait expires
// lets its copies land, sets *expired (the launching plan's or workspace's word) and returns
// (the host reports DGT_ERR_TIMEOUT).
// ------------------------------------------------------------------------------------
__device__ __forceinline__ void note_expired(unsigned int* expired) {
    *reinterpret_cast<volatile unsigned int*>(expired) = 1u;
    __threadfence_system();
}

template <int N, bool ZGT>
__global__ void __launch_bounds__(AdjCfg<float, N>::THREADS, AdjCfg<float, N>::MINB)
    fft_prod_adj_tma_p2(const __grid_constant__ CUtensorMap ymap, const __grid_constant__ CUtensorMap zgmap,
                        const float2* __restrict__ zg, float2* __restrict__ zf, SepGeom g, int64_t J,
                        const float2* __restrict__ tw, long long wait_limit, unsigned int* expired) {
    using C = float2;
    using CF = AdjCfg<float, N>;
    constexpr int W = CF::W;
    constexpr int G = Pow2<N>::G;
    constexpr int BOXR = N < 256 ? N : 256;
    constexpr int NB = N / BOXR;
    constexpr uint32_t STAGE = (uint32_t)(N * W * sizeof(C));
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* stage = reinterpret_cast<C*>(smem_raw);
    C* sm = reinterpret_cast<C*>(smem_raw + 2 * STAGE);
    uint64_t* barY = reinterpret_cast<uint64_t*>(smem_raw + 2 * STAGE + CF::SMEM);
    uint64_t* barZ = barY + 2;
    const int c = threadIdx.x % W, t = threadIdx.x / W;
    const int64_t b = blockIdx.y;
    const int k0 = blockIdx.x * W;
    const int64_t k = k0 + c;
    const bool ok = k < g.M;
    const int q = (int)g.q;
    const int iters = (int)J * q;
    const float scale = 1.f / (float)N;
    if (threadIdx.x == 0) {
        mbar_init(barY, 1);
        mbar_init(barY + 1, 1);
        mbar_init(barZ, 1);
        mbar_init(barZ + 1, 1);
        mbar_fence_init();
    }
    __syncthreads();
    // Y tile of iteration it = (j, w): rows w + q nu of Y[b][j], columns k0 .. k0 + W - 1
    auto issue_y = [&](int it) {
        const int j = it / q, w = it % q, s = it & 1;
        mbar_arrive_expect_tx(barY + s, STAGE);
        for (int i = 0; i < NB; ++i)
            tma_load_3d(stage + (size_t)s * N * W + (size_t)i * BOXR * W, &ymap, k0, w,
                        (int)((b * J + j) * N) + i * BOXR, barY + s);
    };
    // window factor tile of iteration it: rows xi of ZG~_j, columns k0 - a w (+ K0), into the
    // buffer whose Y tile has just been read
    auto issue_z = [&](int it) {
        const int j = it / q, w = it % q, s = it & 1;
        int64_t col0 = k0 - g.a * w;
        if (col0 < 0) col0 += g.K0;
        mbar_arrive_expect_tx(barZ + s, STAGE);
        for (int i = 0; i < NB; ++i)
            tma_load_3d(stage + (size_t)s * N * W + (size_t)i * BOXR * W, &zgmap, (int)col0, 0, j * N + i * BOXR,
                        barZ + s);
    };
    // the copies of this CTA still in flight land before its shared memory is released
    auto drain = [&](int it, bool y_now, bool z_now) {
        const uint32_t ph = (uint32_t)((it >> 1) & 1);
        if (y_now) mbar_wait(barY + (it & 1), ph, kWaitCycles);
        if (z_now) mbar_wait(barZ + (it & 1), ph, kWaitCycles);
        if (it + 1 < iters) mbar_wait(barY + ((it + 1) & 1), (uint32_t)(((it + 1) >> 1) & 1), kWaitCycles);
    };
    if (threadIdx.x == 0) {
        issue_y(0);
        if constexpr (ZGT) {
            if (iters > 1) issue_y(1);
        }
    }
    C acc[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) acc[i] = mk(0.f, 0.f);
    for (int it = 0; it < iters; ++it) {
        const int s = it & 1;
        const uint32_t ph = (uint32_t)((it >> 1) & 1);
        const int j = it / q, w = it % q;
        const C* tile = stage + (size_t)s * N * W;
        C v[16];
        if constexpr (ZGT) {
            const bool late = wait_limit == 0 || !mbar_wait(barY + s, ph, wait_limit);
#pragma unroll
            for (int m = 0; m < 16; ++m) v[m] = tile[(t + G * m) * W + c];
            if (__syncthreads_or(late)) {         // also: every thread has read its Y values
                if (threadIdx.x == 0) {
                    note_expired(expired);
                    drain(it, true, false);
                }
                return;
            }
            if (threadIdx.x == 0) issue_z(it);
            fft_p2_regs<N, -1, W, false>(c, t, sm, tw, v);
        } else {
            // buffer s ^ 1 was last read in iteration it - 1, before that iteration's final barrier
            if (threadIdx.x == 0 && it + 1 < iters) issue_y(it + 1);
            const bool late = wait_limit == 0 || !mbar_wait(barY + s, ph, wait_limit);
            if (__syncthreads_or(late)) {
                if (threadIdx.x == 0) {
                    note_expired(expired);
                    drain(it, true, false);
                }
                return;
            }
            fft_p2<N, -1, W, false>(c, t, sm, tw, [&](int nu) -> C { return tile[nu * W + c]; }, v);
        }
        int64_t colG = k - g.a * w;
        const bool wrap = colG < 0;
        if (wrap) colG += g.K0;
        bool lateZ = false;
        if constexpr (ZGT) lateZ = wait_limit == 0 || !mbar_wait(barZ + s, ph, wait_limit);
        if (ok && !lateZ) {
            const C* zgj = zg + j * g.L + colG;
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int xi = p2_out_pos<N>(t, i);
                C zv;
                if constexpr (ZGT) zv = tile[xi * W + c];
                else zv = zgj[(int64_t)xi * g.K0];
                C u = cmul(cscale(v[i], scale), zv);
                if (wrap) u = cmul(u, __ldg(tw + xi));
                acc[i] = cadd(acc[i], u);
            }
        }
        // the exchange buffer and buffer s are reused
        if constexpr (ZGT) {
            if (__syncthreads_or(lateZ)) {
                if (threadIdx.x == 0) {
                    note_expired(expired);
                    drain(it, false, true);
                }
                return;
            }
            if (threadIdx.x == 0 && it + 2 < iters) issue_y(it + 2);
        } else {
            __syncthreads();
        }
    }
    if (ok) {
#pragma unroll
        for (int i = 0; i < 16; ++i) zf[b * g.L + (int64_t)p2_out_pos<N>(t, i) * g.K0 + k] = acc[i];
    }
}

// ------------------------------------------------------------------------------------
// Fused Zak analysis (p = 1, so K0 = L/d = M and the Zak columns are the product columns).
// zak_prod_ifft: one CTA per tile of W columns k computes the Zak DFT of the signal columns
// (zak_fwd), keeps ZF[.][k] in registers, and for every (j, w) forms ZF conj(ZG~_j[.][k - a w]),
// transforms it back over xi and stores Y[b][j][w + q nu][k] / d (prod_ifft): ZF never goes
// to memory and is read once instead of J q times.   grid (k-tiles, B)
// (The adjoint pair fft_prod_adj + zak_inv stays two kernels: fused, the inverse Zak DFT ran
// at the accumulating kernel's occupancy and the pair got slower.)  Its transforms keep the
// scalar complex additions: with the packed ones it ran 3 % slower despite fewer instructions.
// ------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(ColCfg<T, N>::THREADS) zak_prod_ifft_p2(const void* __restrict__ src, int src_real,
                                                                          int64_t sbs, const cplx<T>* __restrict__ zg,
                                                                          int64_t J, cplx<T>* __restrict__ y, SepGeom g,
                                                                          const cplx<T>* __restrict__ tw,
                                                                          ChirpParams<cplx<T>> pre) {
    using C = cplx<T>;
    using CF = ColCfg<T, N>;
    constexpr int G = Pow2<N>::G;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.y;
    const int64_t k = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = k < g.M;
    const int64_t K0 = g.K0;
    // the Zak column, scaled once by 1 / d (a power of two, so exactly as the products would be)
    const T scale = (T)1 / (T)N;
    C zfm[16];
    {
        C v[16];
        fft_p2<N, -1, CF::W, false, false>(c, t, sm, tw, [&](int e) -> C {
            if (!ok) return mk((T)0, (T)0);
            const int64_t l = k + K0 * e;
            C x = load_any<C>(src, src_real, b * sbs + l);
            if (pre.mode == PRE_CHIRP) x = cmul(x, chirp_factor(pre, l));
            return x;
        }, v);
#pragma unroll
        for (int i = 0; i < 16; ++i) zfm[p2_out_m<N>(i)] = cscale(v[i], scale);
    }
    const int64_t ystride = g.q * g.M;                     // Y rows w + q nu, nu = 0, 1, ...
    for (int64_t j = 0; j < J; ++j) {
        for (int64_t w = 0; w < g.q; ++w) {
            int64_t colG = k - g.a * w;
            const bool wrap = colG < 0;
            if (wrap) colG += K0;
            const C* zgj = zg + j * g.L + colG;
            C v[16];
#pragma unroll
            for (int m = 0; m < 16; ++m) {
                const int xi = t + G * m;
                C x = ok ? cmulc(zfm[m], zgj[(int64_t)xi * K0]) : mk((T)0, (T)0);
                if (wrap) x = cmulc(x, __ldg(tw + xi));
                v[m] = x;
            }
            fft_p2_regs<N, +1, CF::W, false, false>(c, t, sm, tw, v);
            if (ok) {
                C* yb = y + ((b * J + j) * g.d * g.q + w) * g.M + k;
#pragma unroll
                for (int i = 0; i < 16; ++i) yb[(int64_t)p2_out_pos<N>(t, i) * ystride] = v[i];
            }
        }
    }
}

// ------------------------------------------------------------------------------------
// zak_inv: unnormalised inverse DFT over xi per column, post-op, store
// ------------------------------------------------------------------------------------
template <typename T, int N>
__global__ void __launch_bounds__(ColCfg<T, N>::THREADS) zak_inv_p2(const cplx<T>* __restrict__ zf, int64_t zbs,
                                                                    void* __restrict__ dst, int dst_real, int64_t dbs,
                                                                    int64_t K0, const cplx<T>* __restrict__ tw,
                                                                    ChirpParams<cplx<T>> post, T scale) {
    using C = cplx<T>;
    using CF = ColCfg<T, N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw);
    const int c = threadIdx.x % CF::W, t = threadIdx.x / CF::W;
    const int64_t b = blockIdx.y;
    const int64_t col = (int64_t)blockIdx.x * CF::W + c;
    const bool ok = col < K0;
    C v[16];
    fft_p2<N, +1, CF::W>(c, t, sm, tw, [&](int xi) -> C {
        return ok ? zf[b * zbs + (int64_t)xi * K0 + col] : mk((T)0, (T)0);
    }, v);
    if (ok) {
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int64_t l = col + K0 * p2_out_pos<N>(t, i);
            C x = cscale(v[i], scale);
            if (post.mode == PRE_CHIRP) x = cmul(x, chirp_factor(post, l));
            store_any(dst, dst_real, b * dbs + l, x);
        }
    }
}

// ------------------------------------------------------------------------------------
// row kernels: per-row state of the route post-processing
// ------------------------------------------------------------------------------------
template <typename C> struct RowMap {
    int64_t base;      // offset of output channel 0 of this row (modes with a per-row phase)
    int64_t rot;       // cyclic rotation of the channel index (shear, s0 = 0)
    C ph;              // per-row phase
};

template <typename C>
__device__ __forceinline__ RowMap<C> row_map(const PostParams<C>& pp, const SepGeom& g, int64_t b, int64_t j,
                                             int64_t nn) {
    RowMap<C> r;
    const int64_t o0 = out_index(pp, g, b, j, nn, 0, r.ph);
    if (pp.mode == POST_SHEAR0) {
        r.base = (b * pp.N + nn) * pp.M;
        r.rot = o0 - r.base;
    } else {
        r.base = o0;
        r.rot = 0;
    }
    return r;
}

// fft_post: FFT over k of rows of Y, route post-processing, store into c.  SH1 selects the
// per-coefficient index map of the frequency-shear branch; the other modes need one
// (base, rotation, phase) per row, computed before the transform so that it is not live
// beside the 16 values.  Separate instantiations keep the register budget of each.
template <typename T, int N, bool SH1, bool HALF>
__global__ void __launch_bounds__(RowCfg<N>::THREADS) fft_post_p2(const cplx<T>* __restrict__ y,
                                                                  cplx<T>* __restrict__ c, SepGeom g, int64_t J,
                                                                  int64_t rows_total, const cplx<T>* __restrict__ tw,
                                                                  PostParams<cplx<T>> pp) {
    using C = cplx<T>;
    using RC = RowCfg<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gi = threadIdx.x / RC::G, t = threadIdx.x % RC::G;
    C* sm = reinterpret_cast<C*>(smem_raw) + gi * Pow2<N>::SMEM;
    const int64_t row = (int64_t)blockIdx.x * RC::RPB + gi;
    const bool ok = row < rows_total;
    const C* yr = y + row * N;
    const int64_t b = ok ? (int64_t)pp.mJN.div((uint64_t)row) : 0;
    const int64_t rem = row - b * (int64_t)pp.mJN.d;
    const int64_t j = ok ? (int64_t)pp.mNs.div((uint64_t)rem) : 0, nn = ok ? rem - j * (int64_t)pp.mNs.d : 0;
    if constexpr (SH1) {
        C v[16];
        fft_p2<N, -1, 1>(0, t, sm, tw, [&](int k) -> C { return ok ? yr[k] : mk((T)0, (T)0); }, v);
        if (!ok) return;
        if (pp.sh1_fast) {
            const Sh1Row sr = sh1_row(pp, b, nn);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                C ph;
                const int64_t o = sh1_at(pp, sr, p2_out_pos<N>(t, i), ph);
                c[o] = cmul(v[i], ph);
            }
            return;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            C ph;
            const int64_t o = out_index(pp, g, b, j, nn, p2_out_pos<N>(t, i), ph);
            c[o] = cmul(v[i], ph);
        }
    } else {
        RowMap<C> rm{};
        if (ok) rm = row_map(pp, g, b, j, nn);
        C v[16];
        fft_p2<N, -1, 1>(0, t, sm, tw, [&](int k) -> C { return ok ? yr[k] : mk((T)0, (T)0); }, v);
        if (!ok) return;
        const int rot = (int)rm.rot;
        if constexpr (HALF) {
            // channels 0..N/2 of output row rm.base / N, rows of N/2 + 1
            C* cb = c + (rm.base / N) * (N / 2 + 1);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int ch = (p2_out_pos<N>(t, i) + rot) & (N - 1);
                if (ch <= N / 2) cb[ch] = cmul(v[i], rm.ph);
            }
        } else {
            C* cb = c + rm.base;
#pragma unroll
            for (int i = 0; i < 16; ++i) cb[(p2_out_pos<N>(t, i) + rot) & (N - 1)] = cmul(v[i], rm.ph);
        }
    }
}

// pre_ifft: gather c with conjugate phases, unnormalised inverse FFT, store rows of Y
template <typename T, int N, bool SH1, bool HALF>
__global__ void __launch_bounds__(RowCfg<N>::THREADS) pre_ifft_p2(const cplx<T>* __restrict__ c,
                                                                  cplx<T>* __restrict__ y, SepGeom g, int64_t J,
                                                                  int64_t rows_total, const cplx<T>* __restrict__ tw,
                                                                  PostParams<cplx<T>> pp) {
    using C = cplx<T>;
    using RC = RowCfg<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gi = threadIdx.x / RC::G, t = threadIdx.x % RC::G;
    C* sm = reinterpret_cast<C*>(smem_raw) + gi * Pow2<N>::SMEM;
    const int64_t row = (int64_t)blockIdx.x * RC::RPB + gi;
    const bool ok = row < rows_total;
    const int64_t b = ok ? (int64_t)pp.mJN.div((uint64_t)row) : 0;
    const int64_t rem = row - b * (int64_t)pp.mJN.d;
    const int64_t j = ok ? (int64_t)pp.mNs.div((uint64_t)rem) : 0, nn = ok ? rem - j * (int64_t)pp.mNs.d : 0;
    C v[16];
    if constexpr (SH1) {
        if (pp.sh1_fast) {
            const Sh1Row sr = sh1_row(pp, b, nn);
            fft_p2<N, +1, 1>(0, t, sm, tw, [&](int m) -> C {
                if (!ok) return mk((T)0, (T)0);
                C ph;
                const int64_t o = sh1_at(pp, sr, m, ph);
                return cmulc(c[o], ph);
            }, v);
        } else {
            fft_p2<N, +1, 1>(0, t, sm, tw, [&](int m) -> C {
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
        if constexpr (HALF) {
            // channel ch > N/2 is the conjugate of channel (-ch - 2 w(n)) mod N of the same column
            const int64_t r_out = ok ? rm.base / N : 0;
            const C* cb = c + r_out * (N / 2 + 1);
            const int64_t n_out = r_out % pp.N;
            const int tw2 = (int)((n_out * pp.lam1) % pp.lam2) * (int)(2 / pp.lam2);
            fft_p2<N, +1, 1>(0, t, sm, tw, [&](int m) -> C {
                if (!ok) return mk((T)0, (T)0);
                const int ch = (m + rot) & (N - 1);
                C x = ch <= N / 2 ? cb[ch] : cconj(cb[(-ch - tw2) & (N - 1)]);
                return cmulc(x, rm.ph);
            }, v);
        } else {
            const C* cb = c + (ok ? rm.base : 0);
            fft_p2<N, +1, 1>(0, t, sm, tw, [&](int m) -> C {
                return ok ? cmulc(cb[(m + rot) & (N - 1)], rm.ph) : mk((T)0, (T)0);
            }, v);
        }
    }
    if (!ok) return;
    C* yr = y + row * N;
#pragma unroll
    for (int i = 0; i < 16; ++i) yr[p2_out_pos<N>(t, i)] = v[i];
}

// FIR analysis: h_n(k) gathered straight from the signal, FFT over k, store column n of c.
// Sample l = ln + t (tap t of column n) enters with the modulated tap mtaps[wn][t]; the
// column constant exp(-2 pi i ln wn / (lam2 M)) multiplies the transformed column.
// SEG: the RPB columns of a CTA are consecutive columns of one signal; their common segment
// of (RPB - 1) a + Lg samples is first copied to shared memory with coalesced loads, and the
// taps are gathered from there.
// MULTI: windows longer than N (several taps per bin).  Float with Lg <= N is held to 64
// registers, the occupancy of the other row kernels.
template <typename T, int N, bool MULTI, bool SEG>
__global__ void __launch_bounds__(AnaCfg<N>::THREADS, sizeof(T) == 4 && !MULTI ? AnaCfg<N>::MINB : 1)
    fir_analysis_p2(const void* __restrict__ f, int f_real, cplx<T>* __restrict__ c, FirParams<cplx<T>> fp,
                    int64_t rows_total, const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using RC = AnaCfg<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gi = threadIdx.x / RC::G, t = threadIdx.x % RC::G;
    C* sm = reinterpret_cast<C*>(smem_raw) + gi * Pow2<N>::SMEM;
    const int64_t row = (int64_t)blockIdx.x * RC::RPB + gi;
    const bool ok = row < rows_total;
    const int64_t b = ok ? (int64_t)fp.mN.div((uint64_t)row) : 0, n = ok ? row - b * fp.N : 0;
    int64_t ln = fp.a * n - fp.center;                        // time of tap 0, in [0, L)
    if (ln < 0) ln += fp.L;
    const int wn = (int)((n * fp.lam1) % fp.lam2);
    const C* mt = fp.mtaps + (int64_t)wn * fp.Lg;
    const int lnm = (int)(ln & (N - 1));
    const int Lg = (int)fp.Lg;
    const T* fr = reinterpret_cast<const T*>(f) + b * fp.L;
    const C* fc = reinterpret_cast<const C*>(f) + b * fp.L;
    const C ph = wn ? fp.cisLM(-(ln * wn)) : mk((T)1, (T)0);       // column constant
    C v[16];
    if constexpr (SEG) {
        // segment of the CTA's first column: samples ln0 + i, i < S (S <= L, host-checked)
        unsigned char* segp = smem_raw + sizeof(C) * (size_t)Pow2<N>::SMEM * RC::RPB;
        const int S = (RC::RPB - 1) * (int)fp.a + Lg;
        int64_t ln0 = ln - (int64_t)gi * fp.a;                   // all columns of the CTA are valid
        if (ln0 < 0) ln0 += fp.L;
        if (f_real) {
            T* seg = reinterpret_cast<T*>(segp);
            for (int i = threadIdx.x; i < S; i += RC::THREADS) {
                int64_t l = ln0 + i;
                if (l >= fp.L) l -= fp.L;
                seg[i] = fr[l];
            }
        } else {
            C* seg = reinterpret_cast<C*>(segp);
            for (int i = threadIdx.x; i < S; i += RC::THREADS) {
                int64_t l = ln0 + i;
                if (l >= fp.L) l -= fp.L;
                seg[i] = fc[l];
            }
        }
        __syncthreads();
        const int off = gi * (int)fp.a;
        const T* segr = reinterpret_cast<const T*>(segp) + off;
        const C* segc = reinterpret_cast<const C*>(segp) + off;
        fft_p2<N, -1, 1>(0, t, sm, tw, [&](int k) -> C {
            const int tap = (k - lnm) & (N - 1);
            if (tap >= Lg) return mk((T)0, (T)0);
            const C m = __ldg(mt + tap);
            if (f_real) {
                const T x = segr[tap];
                return mk(x * m.x, x * m.y);
            }
            return cmul(segc[tap], m);
        }, v);
    } else {
        auto tap_value = [&](int tap) -> C {
            int64_t l = ln + tap;
            if (l >= fp.L) l -= fp.L;
            const C m = __ldg(mt + tap);
            if (f_real) {
                const T x = fr[l];
                return mk(x * m.x, x * m.y);
            }
            return cmul(fc[l], m);
        };
        if constexpr (!MULTI) {
            // Lg <= N: at most one tap per bin, straight-line loads
            fft_p2<N, -1, 1>(0, t, sm, tw, [&](int k) -> C {
                const int tap = (k - lnm) & (N - 1);
                return (ok && tap < Lg) ? tap_value(tap) : mk((T)0, (T)0);
            }, v);
        } else {
            fft_p2<N, -1, 1>(0, t, sm, tw, [&](int k) -> C {
                C h = mk((T)0, (T)0);
                if (!ok) return h;
                for (int tap = (k - lnm) & (N - 1); tap < Lg; tap += N) h = cadd(h, tap_value(tap));
                return h;
            }, v);
        }
    }
    if (!ok) return;
    if (fp.half) {
        C* cr = c + row * (N / 2 + 1);                          // channels 0..N/2 only
#pragma unroll
        for (int i = 0; i < 16; ++i) {
            const int pos = p2_out_pos<N>(t, i);
            if (pos <= N / 2) cr[pos] = wn ? cmul(v[i], ph) : v[i];
        }
        return;
    }
    C* cr = c + row * N;
    if (wn) {
#pragma unroll
        for (int i = 0; i < 16; ++i) cr[p2_out_pos<N>(t, i)] = cmul(v[i], ph);
    } else {
#pragma unroll
        for (int i = 0; i < 16; ++i) cr[p2_out_pos<N>(t, i)] = v[i];
    }
}

// FIR analysis of real signals with a real window on lattices with lambda2 <= 2 (real-input
// pairing).  With delta = w(n) in {0, 1/2} and l = ln + tap, tap = k - lnm (+ N when k < lnm),
// lnm = ln mod N, the modulation exp(-2 pi i tap delta / N) of the FFT input splits into
// e(k) = exp(-2 pi i k delta / N), the column constant exp(2 pi i lnm delta / N) and the sign
// (-1)^[k < lnm] (delta = 1/2): column n's input is a real sequence r_n(k) (the sign folded in)
// times e(k), and its coefficients are R_n(m + delta) times exp(2 pi i lnm delta / N)
// exp(-2 pi i ln delta / N) = (-1)^floor(ln / N) (delta = 1/2) or 1, R_n(mu) =
// sum_k r_n(k) exp(-2 pi i k mu / N).  Two columns n1, n1 + lambda2 of one w share the FFT of
// (r1 + i r2) e(k), whose outputs are Z(m) = R1(m + delta) + i R2(m + delta); a real sequence
// has R(-mu) = conj(R(mu)), so with P(m) = N - 1 - m (delta = 1/2) or -m mod N (delta = 0)
// R1 = (Z(m) + conj(Z(P(m)))) / 2 and R2 = (Z(m) - conj(Z(P(m)))) / 2i, one exchange through
// shared memory apart.  Pair p of a signal holds columns n1 = (p div lambda2) 2 lambda2 +
// p mod lambda2 and n1 + lambda2; a CTA's RPB pairs cover 2 RPB consecutive columns, whose
// common segment of (2 RPB - 1) a + Lg samples is staged in shared memory first.
template <typename T, int N>
__global__ void __launch_bounds__(AnaCfg<N>::THREADS, sizeof(T) == 4 ? AnaCfg<N>::MINB : 1)
    fir_analysis_pair_p2(const T* __restrict__ f, cplx<T>* __restrict__ c, FirParams<cplx<T>> fp,
                         int64_t pairs_total, const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using RC = AnaCfg<N>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int gi = threadIdx.x / RC::G, t = threadIdx.x % RC::G;
    C* sm = reinterpret_cast<C*>(smem_raw) + gi * Pow2<N>::SMEM;
    T* seg = reinterpret_cast<T*>(smem_raw + sizeof(C) * (size_t)Pow2<N>::SMEM * RC::RPB);
    const int lam2 = (int)fp.lam2;
    const int64_t half = fp.N / 2;                              // pairs per signal
    const int64_t P0 = (int64_t)blockIdx.x * RC::RPB;           // the CTA's first pair (same signal for all)
    const int64_t b = P0 / half;
    const int64_t p0 = P0 - b * half;
    const int64_t nmin = (p0 / lam2) * 2 * lam2;                // first column of the CTA
    const int64_t pp = p0 + gi;
    const int64_t n1 = (pp / lam2) * 2 * lam2 + pp % lam2, n2 = n1 + lam2;
    const bool ok = P0 + gi < pairs_total;
    const int Lg = (int)fp.Lg;
    const bool dh = (n1 * fp.lam1) % lam2 != 0;                 // delta = 1/2 (uniform per group)
    // L2 prefetch of the segment of the CTA kAnaAhead CTAs later, so that its staging loads
    // find the signal in L2 (one prefetch per 128-byte line, every address inside its signal)
    {
        constexpr int kAnaAhead = 256;
        const int64_t Pn = P0 + (int64_t)kAnaAhead * RC::RPB;
        if (Pn < pairs_total) {
            const int64_t bn = Pn / half;
            const int64_t pn = Pn - bn * half;
            int64_t ln = fp.a * ((pn / lam2) * 2 * lam2) - fp.center;
            if (ln < 0) ln += fp.L;
            const int S = (2 * RC::RPB - 1) * (int)fp.a + Lg;
            constexpr int PER = 128 / (int)sizeof(T);
            const T* fn = f + bn * fp.L;
            for (int i = threadIdx.x * PER; i < S; i += RC::THREADS * PER) {
                int64_t l = ln + i;
                if (l >= fp.L) l -= fp.L;
                asm volatile("prefetch.global.L2 [%0];" ::"l"(fn + l));
            }
        }
    }
    // segment of the CTA: samples ln(nmin) + i, i < S; eight loads in flight per thread
    {
        const int S = (2 * RC::RPB - 1) * (int)fp.a + Lg;
        int64_t l0 = fp.a * nmin - fp.center;
        if (l0 < 0) l0 += fp.L;
        const T* fr = f + b * fp.L;
        constexpr int U = 8;
        for (int i0 = threadIdx.x; i0 < S; i0 += U * RC::THREADS) {
            T x[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int i = i0 + u * RC::THREADS;
                int64_t l = l0 + i;
                if (l >= fp.L) l -= fp.L;
                x[u] = i < S ? __ldg(fr + l) : (T)0;
            }
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + u * RC::THREADS < S) seg[i0 + u * RC::THREADS] = x[u];
        }
    }
    __syncthreads();
    auto col_time = [&](int64_t n) {
        int64_t ln = fp.a * n - fp.center;
        return ln < 0 ? ln + fp.L : ln;
    };
    const int64_t ln1 = col_time(n1), ln2 = col_time(n2);
    const int lnm1 = (int)(ln1 & (N - 1)), lnm2 = (int)(ln2 & (N - 1));
    const T* s1 = seg + (n1 - nmin) * fp.a;
    const T* s2 = seg + (n2 - nmin) * fp.a;
    const T* h = fp.rtaps;                                      // the real taps, dense
    C v[16];
    fft_p2<N, -1, 1>(0, t, sm, tw, [&](int k) -> C {
        const int tap1 = (k - lnm1) & (N - 1), tap2 = (k - lnm2) & (N - 1);
        T x1 = (T)0, x2 = (T)0;
        if (tap1 < Lg) {
            x1 = s1[tap1] * __ldg(h + tap1);
            if (dh && k < lnm1) x1 = -x1;
        }
        if (tap2 < Lg) {
            x2 = s2[tap2] * __ldg(h + tap2);
            if (dh && k < lnm2) x2 = -x2;
        }
        C z = mk(x1, x2);
        if (dh) z = cmul(z, __ldg(fp.hb + k));
        return z;
    }, v);
    // exchange: every output of the group's transform into its buffer (the transform's last
    // reads of that buffer came before its final barrier)
#pragma unroll
    for (int i = 0; i < 16; ++i) sm[spad(p2_out_pos<N>(t, i))] = v[i];
    __syncthreads();
    if (!ok) return;
    const T g1 = dh && ((ln1 / N) & 1) ? (T)-0.5 : (T)0.5;     // column constants, with the 1/2
    const T g2 = dh && ((ln2 / N) & 1) ? (T)-0.5 : (T)0.5;
    const int64_t rs = fp.half ? N / 2 + 1 : N;
    C* c1 = c + (b * fp.N + n1) * rs;
    C* c2 = c + (b * fp.N + n2) * rs;
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        const int m = p2_out_pos<N>(t, i);
        if (fp.half && m > N / 2) continue;
        const int pm = dh ? N - 1 - m : ((N - m) & (N - 1));
        const C zp = sm[spad(pm)];
        // R1 = (Z + conj(Zp)) / 2,  R2 = (Z - conj(Zp)) / 2i
        c1[m] = mk(g1 * (v[i].x + zp.x), g1 * (v[i].y - zp.y));
        c2[m] = mk(g2 * (v[i].y + zp.y), g2 * (zp.x - v[i].x));
    }
}

// FIR synthesis: per chunk of `cols` consecutive columns, the inverse FFT of each column (times
// the conjugate column constant exp(+2 pi i ln wn / (lam2 M))) is scattered straight from the
// registers into a shared accumulator of the chunk's segment of a (cols - 1) + Lg samples:
// f(ln + t) += row_n[(ln + t) mod M] conj(mtaps[wn][t]).  Columns D = ceil(Lg / a) apart never
// touch the same sample, so the columns are taken in D rounds (r = q, q + D, ...): within a
// round no two columns collide, and a barrier separates the rounds.  Real output accumulates
// the real part only.  The first and last Lg - a samples of the segment, shared with the
// neighbouring chunks, go to the seam buffer (fir_seams sums them); Lg <= M (one tap per bin).
// RPB columns are transformed at once (RPB groups of N/16 threads): the largest count for 512
// threads, or a quarter of it (float chunks of 16+ columns in ~32 KB, and wherever the wider
// tiles of a larger element do not fit otherwise)
template <int N, int DIV = 1> struct SynCfg {
    static constexpr int G = N / 16;
    static constexpr int RPB0 = G >= 512 ? 1 : 512 / G;
    static constexpr int RPB = RPB0 / DIV > 0 ? RPB0 / DIV : 1;
    static constexpr int THREADS = RPB * G;
};

// MTS: the modulated taps (lam2 Lg values) are first copied to shared memory, after the
// accumulator, and read from there in the scatter.
template <typename T, int N, bool REAL, int DIV, bool MTS = false>
__global__ void __launch_bounds__(SynCfg<N, DIV>::THREADS) fir_synthesis_p2(const cplx<T>* __restrict__ c,
                                                                       void* __restrict__ f,
                                                                       cplx<T>* __restrict__ seams,
                                                                       FirParams<cplx<T>> fp,
                                                                       const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using A = typename std::conditional<REAL, T, C>::type;
    using RC = SynCfg<N, DIV>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw) + (threadIdx.x / RC::G) * Pow2<N>::SMEM;
    A* acc = reinterpret_cast<A*>(smem_raw + sizeof(C) * (size_t)Pow2<N>::SMEM * RC::RPB);
    const int gi = threadIdx.x / RC::G, t = threadIdx.x % RC::G;
    const int64_t b = blockIdx.y;
    const int64_t chunk = blockIdx.x;
    const int64_t nchunks = gridDim.x;
    const int64_t n0 = chunk * fp.cols;
    const int nc = (int)fp.cols;
    const int a = (int)fp.a, Lg = (int)fp.Lg;
    const int S = a * (nc - 1) + Lg;
    const int D = (Lg + a - 1) / a;                  // columns closer than D overlap
    const int PR = nc / D;                           // columns per round (nc % D == 0, host-checked)
    for (int i = threadIdx.x; i < S; i += RC::THREADS) {
        if constexpr (REAL) acc[i] = (T)0;
        else acc[i] = mk((T)0, (T)0);
    }
    const C* mtab = fp.mtaps;
    if constexpr (MTS) {
        C* smt = reinterpret_cast<C*>(
            smem_raw + ((sizeof(C) * (size_t)Pow2<N>::SMEM * RC::RPB + sizeof(A) * (size_t)S + 15) & ~(size_t)15));
        for (int i = threadIdx.x; i < (int)fp.lam2 * Lg; i += RC::THREADS) smt[i] = fp.mtaps[i];
        mtab = smt;
    }
    __syncthreads();
    for (int q = 0; q < D; ++q) {
        for (int s0 = 0; s0 < PR; s0 += RC::RPB) {
            const int sidx = s0 + gi;
            const bool ok = sidx < PR;
            const int r = q + D * sidx;
            const int64_t n = n0 + (ok ? r : 0);
            C v[16];
            if (fp.half) {
                // channel m > N/2 is the conjugate of channel (-m - 2 w(n)) mod N
                const C* cr = c + (b * fp.N + n) * (N / 2 + 1);
                const int tw2 = (int)((n * fp.lam1) % fp.lam2) * (int)(2 / fp.lam2);
                fft_p2<N, +1, 1>(0, t, sm, tw, [&](int m) -> C {
                    if (!ok) return mk((T)0, (T)0);
                    return m <= N / 2 ? cr[m] : cconj(cr[(-m - tw2) & (N - 1)]);
                }, v);
            } else {
                const C* cr = c + (b * fp.N + n) * fp.M;
                fft_p2<N, +1, 1>(0, t, sm, tw, [&](int m) -> C { return ok ? cr[m] : mk((T)0, (T)0); }, v);
            }
            if (ok) {
                const int wn = (int)((n * fp.lam1) % fp.lam2);
                int64_t ln = fp.a * n - fp.center;
                if (ln < 0) ln += fp.L;
                const int lnm = (int)(ln & (N - 1));
                const C ph = wn ? fp.cisLM(ln * wn) : mk((T)1, (T)0);
                const C* mt = mtab + (int64_t)wn * Lg;
                A* ar = acc + r * a;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int tap = (p2_out_pos<N>(t, i) - lnm) & (N - 1);
                    if (tap < Lg) {
                        const C u = wn ? cmul(v[i], ph) : v[i];
                        C m;
                        if constexpr (MTS) m = mt[tap];
                        else m = __ldg(mt + tap);
                        if constexpr (REAL) ar[tap] += u.x * m.x + u.y * m.y;
                        else ar[tap] = cadd(ar[tap], cmulc(u, m));
                    }
                }
            }
        }
        __syncthreads();                            // the next round's columns overlap these
    }
    const int ov = Lg > a ? Lg - a : 0;
    int64_t lstart = fp.a * n0 - fp.center;
    if (lstart < 0) lstart += fp.L;
    // seams of a real output are stored real
    A* seamL = reinterpret_cast<A*>(seams) + (b * nchunks + chunk) * 2 * ov;
    A* seamR = seamL + ov;
    for (int tt = threadIdx.x; tt < S; tt += RC::THREADS) {
        int64_t l = lstart + tt;
        if (l >= fp.L) l -= fp.L;
        const A val = acc[tt];
        if (tt < ov) seamL[tt] = val;
        else if (tt >= S - ov) seamR[tt - (S - ov)] = val;
        else reinterpret_cast<A*>(f)[b * fp.L + l] = val;
    }
}

// FIR synthesis with real output, real window, lambda2 <= 2 (real-output pairing).  With
// delta = w(n) and tap = k - lnm (+ N when k < lnm), column n adds to f(ln + tap)
//   h(tap) sigma_n (-1)^[k < lnm] q_n(k),   q_n(k) = Re sum_m c(m) exp(2 pi i k (m + delta) / N),
// sigma_n = (-1)^floor(ln / N) when delta = 1/2, else 1 (the column constant and the tap
// modulation combined, as in the paired analysis).  q_n is the transform of the Hermitian
// part H(m) = (c(m) + conj(c(P(m)))) / 2, P(m) = N - 1 - m (delta = 1/2) or -m mod N, which is
// real; so two columns of one w share the inverse FFT of H1 + i H2, times
// exp(2 pi i k delta / N): its real part is q1, its imaginary part q2.  (Half rows of a real
// signal's coefficients are already Hermitian: H is the expanded row.)  The pairs are columns
// of rounds q and q + lambda2 (D = ceil(Lg / a), D a multiple of 2 lambda2, so both columns
// of a pair have the same w); the first columns of all groups are scattered, a barrier, then
// the second ones, a barrier (columns of one round never share a sample).
template <typename T, int N, int DIV>
__global__ void __launch_bounds__(SynCfg<N, DIV>::THREADS) fir_synthesis_pair_p2(const cplx<T>* __restrict__ c,
                                                                            T* __restrict__ f,
                                                                            T* __restrict__ seams,
                                                                            FirParams<cplx<T>> fp,
                                                                            const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using RC = SynCfg<N, DIV>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* sm = reinterpret_cast<C*>(smem_raw) + (threadIdx.x / RC::G) * Pow2<N>::SMEM;
    T* acc = reinterpret_cast<T*>(smem_raw + sizeof(C) * (size_t)Pow2<N>::SMEM * RC::RPB);
    const int gi = threadIdx.x / RC::G, t = threadIdx.x % RC::G;
    const int64_t b = blockIdx.y;
    const int64_t chunk = blockIdx.x;
    const int64_t nchunks = gridDim.x;
    const int64_t n0 = chunk * fp.cols;
    const int nc = (int)fp.cols;
    const int a = (int)fp.a, Lg = (int)fp.Lg, lam2 = (int)fp.lam2;
    const int S = a * (nc - 1) + Lg;
    const int D = (Lg + a - 1) / a;
    const int PR = nc / D;                           // columns per round
    // the real taps (real parts of row wn = 0 of the modulated taps, dense), read through L1
    const T* h = fp.rtaps;
    for (int i = threadIdx.x; i < S; i += RC::THREADS) acc[i] = (T)0;
    __syncthreads();
    for (int dq = 0; dq < D / 2; ++dq) {
        const int q1 = (dq / lam2) * 2 * lam2 + dq % lam2;
        for (int s0 = 0; s0 < PR; s0 += RC::RPB) {
            const int sidx = s0 + gi;
            const bool ok = sidx < PR;
            const int r1 = q1 + D * (ok ? sidx : 0), r2 = r1 + lam2;
            const int64_t n1 = n0 + r1, n2 = n0 + r2;
            const bool dh = (n1 * fp.lam1) % lam2 != 0;
            C v[16];
            if (fp.half) {
                const C* c1 = c + (b * fp.N + n1) * (N / 2 + 1);
                const C* c2 = c + (b * fp.N + n2) * (N / 2 + 1);
                const int s2 = dh ? 1 : 0;           // channel m > N/2 is conj of channel (-m - 2 w) mod N
                fft_p2<N, +1, 1>(0, t, sm, tw, [&](int m) -> C {
                    if (!ok) return mk((T)0, (T)0);
                    const C h1 = m <= N / 2 ? c1[m] : cconj(c1[(-m - s2) & (N - 1)]);
                    const C h2 = m <= N / 2 ? c2[m] : cconj(c2[(-m - s2) & (N - 1)]);
                    return mk(h1.x - h2.y, h1.y + h2.x);
                }, v);
            } else {
                const C* c1 = c + (b * fp.N + n1) * N;
                const C* c2 = c + (b * fp.N + n2) * N;
                fft_p2<N, +1, 1>(0, t, sm, tw, [&](int m) -> C {
                    if (!ok) return mk((T)0, (T)0);
                    const int pm = dh ? N - 1 - m : ((N - m) & (N - 1));
                    const C a1 = c1[m], p1 = c1[pm], a2 = c2[m], p2 = c2[pm];
                    // H1 + i H2, H = (c(m) + conj(c(P(m)))) / 2
                    return mk((T)0.5 * ((a1.x + p1.x) - (a2.y - p2.y)), (T)0.5 * ((a1.y - p1.y) + (a2.x + p2.x)));
                }, v);
            }
            int64_t ln1 = fp.a * n1 - fp.center, ln2 = fp.a * n2 - fp.center;
            if (ln1 < 0) ln1 += fp.L;
            if (ln2 < 0) ln2 += fp.L;
            const int lnm1 = (int)(ln1 & (N - 1)), lnm2 = (int)(ln2 & (N - 1));
            const T sg1 = dh && ((ln1 / N) & 1) ? (T)-1 : (T)1;
            const T sg2 = dh && ((ln2 / N) & 1) ? (T)-1 : (T)1;
            if (dh) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const C e = __ldg(fp.hb + p2_out_pos<N>(t, i));      // exp(-pi i k / N)
                    v[i] = mk(v[i].x * e.x + v[i].y * e.y, v[i].y * e.x - v[i].x * e.y);
                }
            }
            {
                // the rows of this group's next pair into L2 while the current pair is scattered
                int dq2 = dq, s2i = s0 + RC::RPB;
                if (s2i >= PR) { s2i = 0; ++dq2; }
                const int sidx2 = s2i + gi;
                if (dq2 < D / 2 && sidx2 < PR) {
                    const int q2 = (dq2 / lam2) * 2 * lam2 + dq2 % lam2;
                    const int64_t m1 = n0 + q2 + D * sidx2;
                    const int64_t rs = fp.half ? N / 2 + 1 : N;
                    const char* r1p = reinterpret_cast<const char*>(c + (b * fp.N + m1) * rs);
                    const char* r2p = reinterpret_cast<const char*>(c + (b * fp.N + m1 + lam2) * rs);
                    const int64_t lines = (rs * (int64_t)sizeof(C) + 127) / 128;
                    for (int64_t li = t; li < lines; li += RC::G) {
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(r1p + li * 128));
                        asm volatile("prefetch.global.L2 [%0];" ::"l"(r2p + li * 128));
                    }
                }
            }
            if (ok) {
                T* ar = acc + r1 * a;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int k = p2_out_pos<N>(t, i);
                    const int tap = (k - lnm1) & (N - 1);
                    if (tap < Lg) ar[tap] += ((dh && k < lnm1) ? -sg1 : sg1) * __ldg(h + tap) * v[i].x;
                }
            }
            __syncthreads();                        // columns of the rounds q and q + lambda2 overlap
            if (ok) {
                T* ar = acc + r2 * a;
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int k = p2_out_pos<N>(t, i);
                    const int tap = (k - lnm2) & (N - 1);
                    if (tap < Lg) ar[tap] += ((dh && k < lnm2) ? -sg2 : sg2) * __ldg(h + tap) * v[i].y;
                }
            }
            __syncthreads();
        }
    }
    const int ov = Lg > a ? Lg - a : 0;
    int64_t lstart = fp.a * n0 - fp.center;
    if (lstart < 0) lstart += fp.L;
    T* seamL = seams + (b * nchunks + chunk) * 2 * ov;
    T* seamR = seamL + ov;
    for (int tt = threadIdx.x; tt < S; tt += RC::THREADS) {
        int64_t l = lstart + tt;
        if (l >= fp.L) l -= fp.L;
        const T val = acc[tt];
        if (tt < ov) seamL[tt] = val;
        else if (tt >= S - ov) seamR[tt - (S - ov)] = val;
        else f[b * fp.L + l] = val;
    }
}

// ------------------------------------------------------------------------------------
// launchers (N dispatched at run time)
// ------------------------------------------------------------------------------------
#define P2_SWITCH(NV, CALL)                    \
    switch (NV) {                              \
        case 128: { constexpr int NN = 128; CALL; } \
        case 256: { constexpr int NN = 256; CALL; } \
        case 512: { constexpr int NN = 512; CALL; } \
        case 1024: { constexpr int NN = 1024; CALL; } \
        case 2048: { constexpr int NN = 2048; CALL; } \
        case 4096: { constexpr int NN = 4096; CALL; } \
        case 8192: { constexpr int NN = 8192; CALL; } \
        default: return cudaErrorNotSupported;  \
    }

// Row transforms (one length-M FFT per coefficient column) also come in N = 16384 for float:
// 1024 threads, 139 KB of shared memory per transform.  Float64 rows of that length do not
// fit one CTA's shared memory.
#define P2_SWITCH_ROWS(NV, CALL)                                                         \
    if ((NV) == 16384) {                                                                 \
        if constexpr (sizeof(T) == 4) { constexpr int NN = 16384; CALL; }                \
        else return cudaErrorNotSupported;                                               \
    }                                                                                    \
    P2_SWITCH(NV, CALL)

inline bool p2_len_ok(int64_t n) { return n >= 128 && n <= 8192 && (n & (n - 1)) == 0; }

template <typename T, int N>
cudaError_t p2_zak_fwd_n(const void* src, int src_real, int64_t sbs, cplx<T>* zf, int64_t zbs, int64_t K0,
                         const void* tw, const ChirpParams<cplx<T>>& pre, int64_t B, cudaStream_t st) {
    using CF = ColCfg<T, N>;
    auto k = zak_fwd_p2<T, N>;
    cudaError_t e = p2_smem(k, CF::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((K0 + CF::W - 1) / CF::W), (unsigned)B);
    k<<<grid, CF::THREADS, CF::SMEM, st>>>(src, src_real, sbs, zf, zbs, K0, (const cplx<T>*)tw, pre);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t p2_prod_ifft_n(const cplx<T>* zf, const cplx<T>* zg, int64_t J, cplx<T>* y, const SepGeom& g,
                           const void* tw, int64_t B, cudaStream_t st) {
    using CF = ColCfg<T, N>;
    auto k = prod_ifft_p2<T, N>;
    cudaError_t e = p2_smem(k, CF::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.M + CF::W - 1) / CF::W), (unsigned)(J * g.q), (unsigned)B);
    k<<<grid, CF::THREADS, CF::SMEM, st>>>(zf, zg, y, g, J, (const cplx<T>*)tw);
    return cudaGetLastError();
}

// cuTensorMapEncodeTiled through the runtime's driver entry point (no link to the driver
// library); null when the driver does not offer it
using TensorMapEncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                          const cuuint64_t*, const cuuint32_t*, const cuuint32_t*,
                                          CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                          CUtensorMapFloatOOBfill);
inline TensorMapEncodeTiled tensor_map_encoder() {
    static const TensorMapEncodeTiled fn = [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess)
            return (TensorMapEncodeTiled) nullptr;
        return (TensorMapEncodeTiled)p;
    }();
    return fn;
}

// Y (rows (b J + j) d q + w + q nu, M columns) as a rank-3 tensor of 8-byte elements:
// (k, w, (b J + j) d + nu) with strides (8, 8 M, 8 q M) bytes; L2 fills of 128 bytes (1.90 ms
// against 2.00 ms with 64-byte fills on 64 audio signals; full-width tiles of 8 columns with
// one CTA per SM: 1.97 ms).  cudaErrorNotSupported when the
// geometry is outside what the tile copies take (odd M, coordinates past 2^31, no encoder).
template <int N>
cudaError_t p2_fft_prod_adj_tma(const float2* y, const float2* zg, int64_t J, float2* zf, const SepGeom& g,
                                const void* tw, int64_t B, unsigned int* expired, cudaStream_t st) {
    using CF = AdjCfg<float, N>;
    constexpr int W = CF::W;
    constexpr int BOXR = N < 256 ? N : 256;
    static_assert(W * sizeof(float2) % 16 == 0, "tile rows of whole 16-byte units");
    const TensorMapEncodeTiled enc = tensor_map_encoder();
    if (!enc || !expired || g.M % 2 || g.d != N || B * J * N >= ((int64_t)1 << 31) ||
        (reinterpret_cast<uintptr_t>(y) & 15))
        return cudaErrorNotSupported;
    const cuuint32_t box[3] = {(cuuint32_t)W, 1, (cuuint32_t)BOXR};
    const cuuint32_t estr[3] = {1, 1, 1};
    CUtensorMap ymap, zgmap;
    const cuuint64_t ydims[3] = {(cuuint64_t)g.M, (cuuint64_t)g.q, (cuuint64_t)(B * J * N)};
    const cuuint64_t ystrides[2] = {(cuuint64_t)g.M * 8, (cuuint64_t)g.q * g.M * 8};
    if (enc(&ymap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(y), ydims, ystrides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
        return cudaErrorNotSupported;
    // the window factor tiles too when a tile never straddles the wrap (a % W == 0) and rows of
    // ZG~ (K0 columns) start on 16-byte boundaries
    bool zgt = g.a % W == 0 && g.K0 % 2 == 0 && g.L == g.d * g.K0 && J * N < ((int64_t)1 << 31) &&
               !(reinterpret_cast<uintptr_t>(zg) & 15);
    if (zgt) {
        const cuuint64_t zdims[3] = {(cuuint64_t)g.K0, 1, (cuuint64_t)(J * N)};
        const cuuint64_t zstrides[2] = {(cuuint64_t)g.K0 * 8, (cuuint64_t)g.K0 * 8};
        zgt = enc(&zgmap, CU_TENSOR_MAP_DATA_TYPE_UINT64, 3, const_cast<float2*>(zg), zdims, zstrides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
    }
    if (!zgt) zgmap = ymap;                                 // not read
    auto k = zgt ? fft_prod_adj_tma_p2<N, true> : fft_prod_adj_tma_p2<N, false>;
    const size_t smem = 2 * (size_t)N * W * sizeof(float2) + CF::SMEM + 4 * sizeof(uint64_t);
    cudaError_t e = p2_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.M + W - 1) / W), (unsigned)B);
    k<<<grid, CF::THREADS, smem, st>>>(ymap, zgmap, zg, zf, g, J, (const float2*)tw, g_wait_limit_cycles, expired);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t p2_fft_prod_adj_n(const cplx<T>* y, const cplx<T>* zg, int64_t J, cplx<T>* zf, const SepGeom& g,
                              const void* tw, int64_t B, unsigned int* expired, cudaStream_t st) {
    using CF = AdjCfg<T, N>;
    if constexpr (sizeof(T) == 4 && CF::HALVE && CF::W >= 2) {
        const cudaError_t e = p2_fft_prod_adj_tma<N>(y, zg, J, zf, g, tw, B, expired, st);
        if (e != cudaErrorNotSupported) return e;
    }
    auto k = fft_prod_adj_p2<T, N>;
    const size_t smem = CF::SMEM;
    cudaError_t e = p2_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.M + CF::W - 1) / CF::W), (unsigned)B);
    k<<<grid, CF::THREADS, smem, st>>>(y, zg, zf, g, J, (const cplx<T>*)tw);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t p2_zak_inv_n(const cplx<T>* zf, int64_t zbs, void* dst, int dst_real, int64_t dbs, int64_t K0,
                         const void* tw, const ChirpParams<cplx<T>>& post, T scale, int64_t B, cudaStream_t st) {
    using CF = ColCfg<T, N>;
    auto k = zak_inv_p2<T, N>;
    cudaError_t e = p2_smem(k, CF::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((K0 + CF::W - 1) / CF::W), (unsigned)B);
    k<<<grid, CF::THREADS, CF::SMEM, st>>>(zf, zbs, dst, dst_real, dbs, K0, (const cplx<T>*)tw, post, scale);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t p2_fft_post_n(const cplx<T>* y, cplx<T>* c, const SepGeom& g, int64_t J, const void* tw,
                          const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    using RC = RowCfg<N>;
    const size_t smem = sizeof(cplx<T>) * (size_t)Pow2<N>::SMEM * RC::RPB;
    if (pp.half && pp.mode == POST_SHEAR1) return cudaErrorNotSupported;
    auto k = pp.mode == POST_SHEAR1 ? fft_post_p2<T, N, true, false>
                                    : pp.half ? fft_post_p2<T, N, false, true> : fft_post_p2<T, N, false, false>;
    cudaError_t e = p2_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = B * J * g.d * g.q;
    PostParams<cplx<T>> q = pp;
    q.mJN = make_mod((uint64_t)(J * g.d * g.q));
    q.mNs = make_mod((uint64_t)(g.d * g.q));
    k<<<(unsigned)((rows + RC::RPB - 1) / RC::RPB), RC::THREADS, smem, st>>>(y, c, g, J, rows, (const cplx<T>*)tw, q);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t p2_pre_ifft_n(const cplx<T>* c, cplx<T>* y, const SepGeom& g, int64_t J, const void* tw,
                          const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    using RC = RowCfg<N>;
    const size_t smem = sizeof(cplx<T>) * (size_t)Pow2<N>::SMEM * RC::RPB;
    if (pp.half && pp.mode == POST_SHEAR1) return cudaErrorNotSupported;
    auto k = pp.mode == POST_SHEAR1 ? pre_ifft_p2<T, N, true, false>
                                    : pp.half ? pre_ifft_p2<T, N, false, true> : pre_ifft_p2<T, N, false, false>;
    cudaError_t e = p2_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = B * J * g.d * g.q;
    PostParams<cplx<T>> q = pp;
    q.mJN = make_mod((uint64_t)(J * g.d * g.q));
    q.mNs = make_mod((uint64_t)(g.d * g.q));
    k<<<(unsigned)((rows + RC::RPB - 1) / RC::RPB), RC::THREADS, smem, st>>>(c, y, g, J, rows, (const cplx<T>*)tw, q);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t p2_fir_analysis_n(const void* f, int f_real, cplx<T>* c, const FirParams<cplx<T>>& fp, const void* tw,
                              int64_t B, cudaStream_t st) {
    using RC = AnaCfg<N>;
    size_t smem = sizeof(cplx<T>) * (size_t)Pow2<N>::SMEM * RC::RPB;
    {
        // real-input pairing: real signal and window, lambda2 <= 2, whole CTAs of pairs
        const int64_t S2 = (2 * RC::RPB - 1) * fp.a + fp.Lg;
        const size_t seg2 = sizeof(T) * (size_t)S2;
        if (f_real && fp.pairable && fp.rtaps && fp.lam2 <= 2 && RC::RPB % fp.lam2 == 0 && fp.Lg <= N &&
            fp.N % (2 * RC::RPB) == 0 && S2 <= fp.L && smem + seg2 <= kSmemBudget && (fp.lam2 == 1 || fp.hb)) {
            auto k = fir_analysis_pair_p2<T, N>;
            cudaError_t e = p2_smem(k, smem + seg2);
            if (e != cudaSuccess) return e;
            const int64_t pairs = B * fp.N / 2;
            k<<<(unsigned)(pairs / RC::RPB), RC::THREADS, smem + seg2, st>>>((const T*)f, c, fp, pairs,
                                                                            (const cplx<T>*)tw);
            return cudaGetLastError();
        }
    }
    // staged segment: every CTA's columns in one signal, the segment shorter than the signal
    const int64_t S = (RC::RPB - 1) * fp.a + fp.Lg;
    const size_t segb = (f_real ? sizeof(T) : sizeof(cplx<T>)) * (size_t)S;
    const bool seg = fp.Lg <= N && fp.N % RC::RPB == 0 && S <= fp.L && smem + segb <= kSmemBudget;
    auto k = fp.Lg > N ? fir_analysis_p2<T, N, true, false>
                       : seg ? fir_analysis_p2<T, N, false, true> : fir_analysis_p2<T, N, false, false>;
    if (seg) smem += segb;
    cudaError_t e = p2_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = B * fp.N;
    k<<<(unsigned)((rows + RC::RPB - 1) / RC::RPB), RC::THREADS, smem, st>>>(f, f_real, c, fp, rows,
                                                                            (const cplx<T>*)tw);
    return cudaGetLastError();
}

// shared bytes of the FIR synthesis kernel for `cols` columns per chunk
template <typename T, int N, int DIV> size_t p2_fir_synthesis_smem(int64_t cols, int64_t a, int64_t Lg, int f_real) {
    return sizeof(cplx<T>) * (size_t)Pow2<N>::SMEM * SynCfg<N, DIV>::RPB +
           (f_real ? sizeof(T) : sizeof(cplx<T>)) * (size_t)(a * (cols - 1) + Lg);
}

// a chunk of `cols` columns suits the variant DIV: rounds of cols / D columns fill whole
// batches of RPB transforms, and the tile (complex accumulator) fits
template <typename T, int N, int DIV> bool p2_fir_synthesis_fits(int64_t cols, int64_t Nn, int64_t a, int64_t Lg) {
    const int64_t D = (Lg + a - 1) / a;
    return Lg <= N && cols % D == 0 && Nn % cols == 0 && (cols / D) % SynCfg<N, DIV>::RPB == 0 &&
           p2_fir_synthesis_smem<T, N, DIV>(cols, a, Lg, 0) <= kSmemBudget;
}

// float: quarter-width CTAs on chunks of at least 16 columns whose tile (real output) takes at
// most 32 KB, about seven CTAs per SM (1.93 ms with half-width, 1.85 ms with quarter-width CTAs
// against 2.08 ms with the full 512-thread CTAs and 64-column chunks, 64 audio signals; chunks
// of 16 columns write 11 % more seam bytes than the coefficients they read)
template <typename T, int N> bool p2_fir_synthesis_small(int64_t cols, int64_t Nn, int64_t a, int64_t Lg) {
    return sizeof(T) == 4 && cols >= 16 && p2_fir_synthesis_fits<T, N, 4>(cols, Nn, a, Lg) &&
           p2_fir_synthesis_smem<T, N, 4>(cols, a, Lg, 1) <= 32 * 1024;
}

template <typename T, int N, int DIV>
cudaError_t p2_fir_synthesis_launch(const cplx<T>* c, void* f, int f_real, cplx<T>* seams,
                                    const FirParams<cplx<T>>& fp, const void* tw, int64_t B, cudaStream_t st) {
    size_t smem = p2_fir_synthesis_smem<T, N, DIV>(fp.cols, fp.a, fp.Lg, f_real);
    dim3 grid((unsigned)(fp.N / fp.cols), (unsigned)B);
    const size_t mtb = sizeof(cplx<T>) * (size_t)(fp.lam2 * fp.Lg);
    if constexpr (sizeof(T) == 4 && DIV == 4) {
        // float quarter-width CTAs: modulated taps from shared memory when they take <= 16 KB
        if (mtb <= 16 * 1024) {
            smem = ((smem + 15) & ~(size_t)15) + mtb;
            auto k = f_real ? fir_synthesis_p2<T, N, true, DIV, true> : fir_synthesis_p2<T, N, false, DIV, true>;
            cudaError_t e = p2_smem(k, smem);
            if (e != cudaSuccess) return e;
            k<<<grid, SynCfg<N, DIV>::THREADS, smem, st>>>(c, f, seams, fp, (const cplx<T>*)tw);
            return cudaGetLastError();
        }
    }
    auto k = f_real ? fir_synthesis_p2<T, N, true, DIV> : fir_synthesis_p2<T, N, false, DIV>;
    cudaError_t e = p2_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<grid, SynCfg<N, DIV>::THREADS, smem, st>>>(c, f, seams, fp, (const cplx<T>*)tw);
    return cudaGetLastError();
}

template <typename T, int N, int DIV>
cudaError_t p2_fir_synthesis_pair_launch(const cplx<T>* c, void* f, cplx<T>* seams, const FirParams<cplx<T>>& fp,
                                         const void* tw, int64_t B, cudaStream_t st) {
    const size_t smem = sizeof(cplx<T>) * (size_t)Pow2<N>::SMEM * SynCfg<N, DIV>::RPB +
                        sizeof(T) * (size_t)(fp.a * (fp.cols - 1) + fp.Lg);
    if (smem > kSmemBudget) return cudaErrorNotSupported;
    auto k = fir_synthesis_pair_p2<T, N, DIV>;
    cudaError_t e = p2_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)(fp.N / fp.cols), (unsigned)B);
    k<<<grid, SynCfg<N, DIV>::THREADS, smem, st>>>(c, (T*)f, (T*)seams, fp, (const cplx<T>*)tw);
    return cudaGetLastError();
}

template <typename T, int N>
cudaError_t p2_fir_synthesis_n(const cplx<T>* c, void* f, int f_real, cplx<T>* seams, const FirParams<cplx<T>>& fp,
                               const void* tw, int64_t B, cudaStream_t st) {
    {
        // real output, real window, lambda2 <= 2, rounds that pair up (D a multiple of 2 lambda2)
        const int64_t D = (fp.Lg + fp.a - 1) / fp.a;
        if (f_real && fp.pairable && fp.rtaps && fp.lam2 <= 2 && fp.Lg <= N && D % (2 * fp.lam2) == 0 && fp.cols % D == 0 &&
            fp.N % fp.cols == 0 && (fp.lam2 == 1 || fp.hb)) {
            cudaError_t e = cudaErrorNotSupported;
            if (p2_fir_synthesis_small<T, N>(fp.cols, fp.N, fp.a, fp.Lg))
                e = p2_fir_synthesis_pair_launch<T, N, 4>(c, f, seams, fp, tw, B, st);
            else if (p2_fir_synthesis_fits<T, N, 1>(fp.cols, fp.N, fp.a, fp.Lg))
                e = p2_fir_synthesis_pair_launch<T, N, 1>(c, f, seams, fp, tw, B, st);
            else if (p2_fir_synthesis_fits<T, N, 4>(fp.cols, fp.N, fp.a, fp.Lg))
                e = p2_fir_synthesis_pair_launch<T, N, 4>(c, f, seams, fp, tw, B, st);
            if (e != cudaErrorNotSupported) return e;
        }
    }
    if (p2_fir_synthesis_small<T, N>(fp.cols, fp.N, fp.a, fp.Lg))
        return p2_fir_synthesis_launch<T, N, 4>(c, f, f_real, seams, fp, tw, B, st);
    if (p2_fir_synthesis_fits<T, N, 1>(fp.cols, fp.N, fp.a, fp.Lg))
        return p2_fir_synthesis_launch<T, N, 1>(c, f, f_real, seams, fp, tw, B, st);
    if (p2_fir_synthesis_fits<T, N, 4>(fp.cols, fp.N, fp.a, fp.Lg))
        return p2_fir_synthesis_launch<T, N, 4>(c, f, f_real, seams, fp, tw, B, st);
    return cudaErrorNotSupported;
}

// columns per chunk for the power-of-two FIR synthesis: the widest chunk (fewest seams) that
// the full-width variant takes, else the widest for the quarter-width one; 0 when neither
// applies (the generic kernel runs)
template <typename T, int N> int64_t p2_fir_synthesis_cols_n(int64_t Nn, int64_t a, int64_t Lg) {
    if (Lg > N) return 0;
    const int64_t D = (Lg + a - 1) / a;
    int64_t best = 0;
    for (int64_t cols = D; cols <= 256; cols += D)
        if (p2_fir_synthesis_small<T, N>(cols, Nn, a, Lg)) best = cols;
    if (best) return best;
    for (int64_t cols = D; cols <= 256; cols += D)
        if (p2_fir_synthesis_fits<T, N, 1>(cols, Nn, a, Lg)) best = cols;
    if (best) return best;
    for (int64_t cols = D; cols <= 256; cols += D)
        if (p2_fir_synthesis_fits<T, N, 4>(cols, Nn, a, Lg)) best = cols;
    return best;
}

template <typename T, int N>
cudaError_t p2_zak_prod_ifft_n(const void* src, int src_real, int64_t sbs, const cplx<T>* zg, int64_t J, cplx<T>* y,
                               const SepGeom& g, const void* tw, const ChirpParams<cplx<T>>& pre, int64_t B,
                               cudaStream_t st) {
    using CF = ColCfg<T, N>;
    auto k = zak_prod_ifft_p2<T, N>;
    cudaError_t e = p2_smem(k, CF::SMEM);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.M + CF::W - 1) / CF::W), (unsigned)B);
    k<<<grid, CF::THREADS, CF::SMEM, st>>>(src, src_real, sbs, zg, J, y, g, (const cplx<T>*)tw, pre);
    return cudaGetLastError();
}

// ------------------------------------------------------------------------------------
// run-time dispatch over the instantiated lengths; cudaErrorNotSupported = use the generic path
// ------------------------------------------------------------------------------------
template <typename T>
cudaError_t p2_zak_fwd(const void* src, int src_real, int64_t sbs, cplx<T>* zf, int64_t zbs, int64_t d, int64_t K0,
                       const void* tw, const ChirpParams<cplx<T>>& pre, int64_t B, cudaStream_t st) {
    P2_SWITCH(d, return (p2_zak_fwd_n<T, NN>(src, src_real, sbs, zf, zbs, K0, tw, pre, B, st)))
}
template <typename T>
cudaError_t p2_prod_ifft(const cplx<T>* zf, const cplx<T>* zg, int64_t J, cplx<T>* y, const SepGeom& g, const void* tw,
                         int64_t B, cudaStream_t st) {
    if (g.p != 1) return cudaErrorNotSupported;
    P2_SWITCH(g.d, return (p2_prod_ifft_n<T, NN>(zf, zg, J, y, g, tw, B, st)))
}
template <typename T>
cudaError_t p2_fft_prod_adj(const cplx<T>* y, const cplx<T>* zg, int64_t J, cplx<T>* zf, const SepGeom& g,
                            const void* tw, int64_t B, unsigned int* expired, cudaStream_t st) {
    if (g.p != 1) return cudaErrorNotSupported;
    P2_SWITCH(g.d, return (p2_fft_prod_adj_n<T, NN>(y, zg, J, zf, g, tw, B, expired, st)))
}
template <typename T>
cudaError_t p2_zak_inv(const cplx<T>* zf, int64_t zbs, void* dst, int dst_real, int64_t dbs, int64_t d, int64_t K0,
                       const void* tw, const ChirpParams<cplx<T>>& post, T scale, int64_t B, cudaStream_t st) {
    P2_SWITCH(d, return (p2_zak_inv_n<T, NN>(zf, zbs, dst, dst_real, dbs, K0, tw, post, scale, B, st)))
}
template <typename T>
cudaError_t p2_zak_prod_ifft(const void* src, int src_real, int64_t sbs, const cplx<T>* zg, int64_t J, cplx<T>* y,
                             const SepGeom& g, const void* tw, const ChirpParams<cplx<T>>& pre, int64_t B,
                             cudaStream_t st) {
    if (g.p != 1 || g.K0 != g.M) return cudaErrorNotSupported;
    P2_SWITCH(g.d, return (p2_zak_prod_ifft_n<T, NN>(src, src_real, sbs, zg, J, y, g, tw, pre, B, st)))
}
template <typename T>
cudaError_t p2_fft_post(const cplx<T>* y, cplx<T>* c, const SepGeom& g, int64_t J, const void* tw,
                        const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    P2_SWITCH_ROWS(g.M, return (p2_fft_post_n<T, NN>(y, c, g, J, tw, pp, B, st)))
}
template <typename T>
cudaError_t p2_pre_ifft(const cplx<T>* c, cplx<T>* y, const SepGeom& g, int64_t J, const void* tw,
                        const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    P2_SWITCH_ROWS(g.M, return (p2_pre_ifft_n<T, NN>(c, y, g, J, tw, pp, B, st)))
}
template <typename T>
cudaError_t p2_fir_analysis(const void* f, int f_real, cplx<T>* c, const FirParams<cplx<T>>& fp, const void* tw,
                            int64_t B, cudaStream_t st) {
    P2_SWITCH(fp.M, return (p2_fir_analysis_n<T, NN>(f, f_real, c, fp, tw, B, st)))
}
template <typename T>
int64_t p2_fir_synthesis_cols(int64_t M, int64_t Nn, int64_t a, int64_t Lg) {
    switch (M) {
        case 128: return p2_fir_synthesis_cols_n<T, 128>(Nn, a, Lg);
        case 256: return p2_fir_synthesis_cols_n<T, 256>(Nn, a, Lg);
        case 512: return p2_fir_synthesis_cols_n<T, 512>(Nn, a, Lg);
        case 1024: return p2_fir_synthesis_cols_n<T, 1024>(Nn, a, Lg);
        case 2048: return p2_fir_synthesis_cols_n<T, 2048>(Nn, a, Lg);
        case 4096: return p2_fir_synthesis_cols_n<T, 4096>(Nn, a, Lg);
        case 8192: return p2_fir_synthesis_cols_n<T, 8192>(Nn, a, Lg);
        default: return 0;
    }
}
template <typename T>
cudaError_t p2_fir_synthesis(const cplx<T>* c, void* f, int f_real, cplx<T>* seams, const FirParams<cplx<T>>& fp,
                             const void* tw, int64_t B, cudaStream_t st) {
    P2_SWITCH(fp.M, return (p2_fir_synthesis_n<T, NN>(c, f, f_real, seams, fp, tw, B, st)))
}

}  // namespace dgt
