// Separable DGT through the Zak / polyphase factorisation, and its adjoint.
//
// Separable lattice (a, M) on Z_L with c = gcd(a,M), p = a/c, q = M/c, d = b/p, K0 = L/d
// (eqs. cd, pq).  For n = w + q nu (w < q, nu < d) and k < M:
//
//   ZF[xi][col]   = sum_{mu<d} f(col + K0 mu) e^{-2 pi i mu xi/d}                (zak_fwd)
//   X_w[xi][k]    = sum_{i<p} ZF[xi][k+iM] conj(ZG~[xi][k+iM-aw])              (prod_ifft)
//   h_n(k)        = (1/d) sum_xi X_w[xi][k] e^{+2 pi i nu xi/d}                    (prod_ifft)
//   c_sep(m, n)   = sum_k h_n(k) e^{-2 pi i k m/M}                                 (fft_post)
//
// ZG~ extends the window's Zak transform to negative columns quasi-periodically,
// ZG~[xi][col-K0] = e^{-2 pi i xi/d} ZG[xi][col].  The three kernels realise the signal
// factorisation, the block products with the inverse FFT over xi, and the channel FFT of
// the flop count in eq. (rect-flops); fft_post also applies the coset phase of eq.
// (mw_phases) or the phase and reindex of Algorithm 1 while storing c(m, n).
//
// Layouts: signals [B][L]; ZF, ZG [.][d][K0] (xi-major); intermediate Y [B][J][N_sep][M_sep]
// (one row per separable time index, k contiguous); coefficients [B][N][M] (m contiguous).
#include "engine.h"
#include "kcommon.cuh"

#include <algorithm>

namespace dgt {


static size_t g_smem_optin = 0;
template <typename K> static cudaError_t prep_smem(K kernel, size_t bytes) {
    if (g_smem_optin == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        g_smem_optin = (size_t)v;
    }
    if (bytes > g_smem_optin) return cudaErrorInvalidValue;
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}


// =====================================================================================
// zak_fwd: column DFTs of length d over the [d][K0] view of each signal
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) zak_fwd_kernel(const void* __restrict__ src, int src_real, int64_t sbs,
                                                              cplx<T>* __restrict__ zf, int64_t zbs, int64_t d,
                                                              int64_t K0, int W, FftPlanDev pl,
                                                              const cplx<T>* __restrict__ tw, ChirpParams<cplx<T>> pre) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int64_t b = blockIdx.y;
    const int64_t col0 = (int64_t)blockIdx.x * W;
    const int nbc = (int)min((int64_t)W, K0 - col0);
    const int total = (int)d * nbc;
    const int TILE = (int)d * W;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = e / nbc, cc = e % nbc;
        const int64_t l = col0 + cc + K0 * i;
        C x = load_any<C>(src, src_real, b * sbs + l);
        if (pre.mode == PRE_CHIRP) x = cmul(x, chirp_factor(pre, l));
        s[i * W + cc] = x;
    }
    __syncthreads();
    const C* r = fft_tile<-1, true>(s, s + TILE, pl, nbc, W, 1, tw);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = e / nbc, cc = e % nbc;
        zf[b * zbs + i * K0 + col0 + cc] = r[i * W + cc];
    }
}

template <typename T>
cudaError_t launch_zak_fwd(const void* src, int src_real, int64_t sbs, cplx<T>* zf, int64_t zbs, int64_t L, int64_t d,
                           const FftRef& fd, const ChirpParams<cplx<T>>& pre, int64_t B, cudaStream_t st) {
    {
        cudaError_t e = p2_zak_fwd<T>(src, src_real, sbs, zf, zbs, d, L / d, fd.tw, pre, B, st);
        if (e != cudaErrorNotSupported) return e;
        e = mr_zak_fwd<T>(src, src_real, sbs, zf, zbs, d, L / d, fd.tw, pre, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    using C = cplx<T>;
    const int64_t K0 = L / d;
    const int64_t cap = tile_cap<T>();
    if (d > cap) return cudaErrorInvalidValue;
    // columns per CTA: a tile of about 48 KB (two buffers), so that several CTAs share an SM
    const int W = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)(24 * 1024 / sizeof(C)) / d, 16, K0}));
    const int thr = threads_for(d * W);
    const size_t smem = 2 * sizeof(C) * (size_t)d * W;
    auto k = zak_fwd_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((K0 + W - 1) / W), (unsigned)B);
    k<<<grid, thr, smem, st>>>(src, src_real, sbs, zf, zbs, d, K0, W, fd.pl, (const C*)fd.tw, pre);
    return cudaGetLastError();
}

// =====================================================================================
// prod_ifft: X_w = sum_i ZF conj(ZG~_j) on a block of k, inverse FFT over xi, / d
// grid (k-blocks, J*q, B)
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) prod_ifft_kernel(const cplx<T>* __restrict__ zf,
                                                                const cplx<T>* __restrict__ zg, cplx<T>* __restrict__ y,
                                                                SepGeom g, int64_t J, int W, FftPlanDev pl,
                                                                const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int64_t b = blockIdx.z;
    const int64_t j = blockIdx.y / g.q, w = blockIdx.y % g.q;
    const int64_t k0 = (int64_t)blockIdx.x * W;
    const int nbc = (int)min((int64_t)W, g.M - k0);
    const int total = (int)g.d * nbc;
    const int TILE = (int)g.d * W;
    const C* zfb = zf + b * g.L;
    const C* zgj = zg + j * g.L;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int xi = e / nbc, kk = e % nbc;
        const int64_t k = k0 + kk;
        C X = mk((T)0, (T)0);
        for (int64_t i = 0; i < g.p; ++i) {
            const int64_t colF = k + i * g.M;
            int64_t colG = colF - g.a * w;
            const bool wrap = colG < 0;
            if (wrap) colG += g.K0;
            C t = cmulc(zfb[xi * g.K0 + colF], zgj[xi * g.K0 + colG]);
            if (wrap) t = cmulc(t, __ldg(tw + xi));
            X = cadd(X, t);
        }
        s[xi * W + kk] = X;
    }
    __syncthreads();
    const C* r = fft_tile<+1, true>(s, s + TILE, pl, nbc, W, 1, tw);
    const T scale = (T)1 / (T)g.d;
    const int64_t Nsep = g.d * g.q;
    C* yb = y + ((b * J + j) * Nsep) * g.M;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int nu = e / nbc, kk = e % nbc;
        yb[(w + g.q * nu) * g.M + k0 + kk] = cscale(r[nu * W + kk], scale);
    }
}

template <typename T>
cudaError_t launch_prod_ifft(const cplx<T>* zf, const cplx<T>* zg, int64_t J, cplx<T>* y, const SepGeom& g,
                             const FftRef& fd, int64_t B, cudaStream_t st) {
    {
        cudaError_t e = p2_prod_ifft<T>(zf, zg, J, y, g, fd.tw, B, st);
        if (e != cudaErrorNotSupported) return e;
        e = mr_prod_ifft<T>(zf, zg, J, y, g, fd.tw, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    using C = cplx<T>;
    const int64_t cap = tile_cap<T>();
    if (g.d > cap) return cudaErrorInvalidValue;
    const int W = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)(24 * 1024 / sizeof(C)) / g.d, 16, g.M}));
    const int thr = threads_for(g.d * W);
    const size_t smem = 2 * sizeof(C) * (size_t)g.d * W;
    auto k = prod_ifft_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.M + W - 1) / W), (unsigned)(J * g.q), (unsigned)B);
    k<<<grid, thr, smem, st>>>(zf, zg, y, g, J, W, fd.pl, (const C*)fd.tw);
    return cudaGetLastError();
}

// =====================================================================================
// fft_post: forward FFT over k of nr rows of Y, then phase / reindex store into c
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) fft_post_kernel(const cplx<T>* __restrict__ y, cplx<T>* __restrict__ c,
                                                               SepGeom g, int64_t J, int64_t rows_total, int R,
                                                               FftPlanDev pl, const cplx<T>* __restrict__ tw,
                                                               PostParams<cplx<T>> pp) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = pl.n;
    const int pitch = n + 1;
    const int64_t row0 = (int64_t)blockIdx.x * R;
    const int nr = (int)min((int64_t)R, rows_total - row0);
    const int total = nr * n;
    const int TILE = R * pitch;
    (void)total;
    for (int r = 0; r < nr; ++r)
        for (int k = threadIdx.x; k < n; k += blockDim.x) s[r * pitch + k] = y[(row0 + r) * n + k];
    __syncthreads();
    s = fft_tile<-1, false>(s, s + TILE, pl, nr, 1, pitch, tw);
    const int64_t Nsep = g.d * g.q;
    for (int r = 0; r < nr; ++r) {
        // the row's separable indices, once per row
        const int64_t row = row0 + r;
        const int64_t b = row / (J * Nsep);
        const int64_t rem = row - b * J * Nsep;
        const int64_t j = rem / Nsep, nn = rem - j * Nsep;
        if (pp.mode == POST_SHEAR1) {
            for (int m = threadIdx.x; m < n; m += blockDim.x) {
                C ph;
                const int64_t o = out_index(pp, g, b, j, nn, m, ph);
                c[o] = cmul(s[r * pitch + m], ph);
            }
            continue;
        }
        // the other modes: output m of the row lands at o0 + m (rotated cyclically for the
        // time shear), all with the phase of m = 0
        C ph;
        const int64_t o0 = out_index(pp, g, b, j, nn, 0, ph);
        if (pp.mode == POST_SHEAR0) {
            // iterate over the output channel so the store is contiguous
            const int64_t base = (b * pp.N + nn) * pp.M;
            const int rot = (int)(o0 - base);
            for (int m = threadIdx.x; m < n; m += blockDim.x) {
                int src = m - rot;
                if (src < 0) src += n;
                c[base + m] = cmul(s[r * pitch + src], ph);
            }
        } else {
            for (int m = threadIdx.x; m < n; m += blockDim.x) c[o0 + m] = cmul(s[r * pitch + m], ph);
        }
    }
}

template <typename T>
cudaError_t launch_fft_post(const cplx<T>* y, cplx<T>* c, const SepGeom& g, int64_t J, const FftRef& fm,
                            const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    {
        cudaError_t e = p2_fft_post<T>(y, c, g, J, fm.tw, pp, B, st);
        if (e != cudaErrorNotSupported) return e;
        e = mr_fft_post<T>(y, c, g, J, fm.tw, pp, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    if (pp.half) return cudaErrorNotSupported;       // half-channel output: power-of-two kernels only
    using C = cplx<T>;
    const int64_t n = g.M;
    const int64_t cap = tile_cap<T>();
    if (n + 1 > cap) return cudaErrorInvalidValue;
    // rows per CTA: a tile of about 48 KB (two buffers), so that several CTAs share an SM
    const int R = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)(24 * 1024 / sizeof(C)) / (n + 1), 16));
    const int thr = threads_for(n * R);
    const size_t smem = 2 * sizeof(C) * (size_t)(n + 1) * R;
    auto k = fft_post_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = B * J * g.d * g.q;
    k<<<(unsigned)((rows + R - 1) / R), thr, smem, st>>>(y, c, g, J, rows, R, fm.pl, (const C*)fm.tw, pp);
    return cudaGetLastError();
}

// =====================================================================================
// pre_ifft (adjoint of fft_post): gather with conjugate phases, unnormalised inverse FFT
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) pre_ifft_kernel(const cplx<T>* __restrict__ c, cplx<T>* __restrict__ y,
                                                               SepGeom g, int64_t J, int64_t rows_total, int R,
                                                               FftPlanDev pl, const cplx<T>* __restrict__ tw,
                                                               PostParams<cplx<T>> pp) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = pl.n;
    const int pitch = n + 1;
    const int64_t row0 = (int64_t)blockIdx.x * R;
    const int nr = (int)min((int64_t)R, rows_total - row0);
    const int total = nr * n;
    const int64_t Nsep = g.d * g.q;
    (void)total;
    for (int r = 0; r < nr; ++r) {
        // the row's separable indices, once per row
        const int64_t row = row0 + r;
        const int64_t b = row / (J * Nsep);
        const int64_t rem = row - b * J * Nsep;
        const int64_t j = rem / Nsep, nn = rem - j * Nsep;
        if (pp.mode == POST_SHEAR1) {
            for (int m = threadIdx.x; m < n; m += blockDim.x) {
                C ph;
                const int64_t o = out_index(pp, g, b, j, nn, m, ph);
                s[r * pitch + m] = cmulc(c[o], ph);
            }
            continue;
        }
        C ph;
        const int64_t o0 = out_index(pp, g, b, j, nn, 0, ph);
        if (pp.mode == POST_SHEAR0) {
            const int64_t base = (b * pp.N + nn) * pp.M;
            const int rot = (int)(o0 - base);
            for (int m = threadIdx.x; m < n; m += blockDim.x) {
                int dst = m - rot;                      // separable channel of output channel m
                if (dst < 0) dst += n;
                s[r * pitch + dst] = cmulc(c[base + m], ph);
            }
        } else {
            for (int m = threadIdx.x; m < n; m += blockDim.x) s[r * pitch + m] = cmulc(c[o0 + m], ph);
        }
    }
    __syncthreads();
    const C* res = fft_tile<+1, false>(s, s + R * pitch, pl, nr, 1, pitch, tw);
    for (int r = 0; r < nr; ++r)
        for (int k = threadIdx.x; k < n; k += blockDim.x) y[(row0 + r) * n + k] = res[r * pitch + k];
}

template <typename T>
cudaError_t launch_pre_ifft(const cplx<T>* c, cplx<T>* y, const SepGeom& g, int64_t J, const FftRef& fm,
                            const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st) {
    {
        cudaError_t e = p2_pre_ifft<T>(c, y, g, J, fm.tw, pp, B, st);
        if (e != cudaErrorNotSupported) return e;
        e = mr_pre_ifft<T>(c, y, g, J, fm.tw, pp, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    if (pp.half) return cudaErrorNotSupported;
    using C = cplx<T>;
    const int64_t n = g.M;
    const int64_t cap = tile_cap<T>();
    if (n + 1 > cap) return cudaErrorInvalidValue;
    // rows per CTA: a tile of about 48 KB (two buffers), so that several CTAs share an SM
    const int R = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)(24 * 1024 / sizeof(C)) / (n + 1), 16));
    const int thr = threads_for(n * R);
    const size_t smem = 2 * sizeof(C) * (size_t)(n + 1) * R;
    auto k = pre_ifft_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    const int64_t rows = B * J * g.d * g.q;
    k<<<(unsigned)((rows + R - 1) / R), thr, smem, st>>>(c, y, g, J, rows, R, fm.pl, (const C*)fm.tw, pp);
    return cudaGetLastError();
}

// =====================================================================================
// fft_prod_adj (adjoint of prod_ifft): for every (j, w) FFT over nu with 1/d, multiply by
// the synthesis window factor and accumulate into ZF'[xi][k + iM]; grid (k-blocks, B)
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) fft_prod_adj_kernel(const cplx<T>* __restrict__ y,
                                                                   const cplx<T>* __restrict__ zg,
                                                                   cplx<T>* __restrict__ zf, SepGeom g, int64_t J,
                                                                   int W, FftPlanDev pl,
                                                                   const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int TILE = (int)g.d * W;
    C* acc = s + 2 * TILE;
    const int64_t b = blockIdx.y;
    const int64_t k0 = (int64_t)blockIdx.x * W;
    const int nbc = (int)min((int64_t)W, g.M - k0);
    const int total = (int)g.d * nbc;
    const int64_t Nsep = g.d * g.q;
    const T scale = (T)1 / (T)g.d;
    for (int e = threadIdx.x; e < total * (int)g.p; e += blockDim.x) acc[e] = mk((T)0, (T)0);
    for (int64_t j = 0; j < J; ++j) {
        const C* yb = y + ((b * J + j) * Nsep) * g.M;
        const C* zgj = zg + j * g.L;
        for (int64_t w = 0; w < g.q; ++w) {
            __syncthreads();
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                const int nu = e / nbc, kk = e % nbc;
                s[nu * W + kk] = yb[(w + g.q * nu) * g.M + k0 + kk];
            }
            __syncthreads();
            const C* r = fft_tile<-1, true>(s, s + TILE, pl, nbc, W, 1, tw);
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                const int xi = e / nbc, kk = e % nbc;
                const int64_t k = k0 + kk;
                const C X = cscale(r[xi * W + kk], scale);
                for (int64_t i = 0; i < g.p; ++i) {
                    int64_t colG = k + i * g.M - g.a * w;
                    const bool wrap = colG < 0;
                    if (wrap) colG += g.K0;
                    C t = cmul(X, zgj[xi * g.K0 + colG]);
                    if (wrap) t = cmul(t, __ldg(tw + xi));
                    acc[i * total + e] = cadd(acc[i * total + e], t);
                }
            }
        }
    }
    __syncthreads();
    C* zfb = zf + b * g.L;
    for (int64_t i = 0; i < g.p; ++i)
        for (int e = threadIdx.x; e < total; e += blockDim.x) {
            const int xi = e / nbc, kk = e % nbc;
            zfb[xi * g.K0 + k0 + kk + i * g.M] = acc[i * total + e];
        }
}

template <typename T>
cudaError_t launch_fft_prod_adj(const cplx<T>* y, const cplx<T>* zg, int64_t J, cplx<T>* zf, const SepGeom& g,
                                const FftRef& fd, int64_t B, unsigned int* expired, cudaStream_t st) {
    {
        cudaError_t e = p2_fft_prod_adj<T>(y, zg, J, zf, g, fd.tw, B, expired, st);
        if (e != cudaErrorNotSupported) return e;
        e = mr_fft_prod_adj<T>(y, zg, J, zf, g, fd.tw, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    using C = cplx<T>;
    // two work tiles d*W plus the accumulator p*d*W
    const int64_t elems = (int64_t)(kSmemBudget / sizeof(C));
    const int64_t W = std::min<int64_t>({std::max<int64_t>(1, (int64_t)(36 * 1024 / sizeof(C)) / (g.d * (2 + g.p))),
                                         elems / (g.d * (2 + g.p)), 16, g.M});
    if (W < 1) return cudaErrorInvalidValue;
    const int thr = threads_for(g.d * W);
    const size_t smem = sizeof(C) * (size_t)g.d * W * (2 + g.p);
    auto k = fft_prod_adj_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.M + W - 1) / W), (unsigned)B);
    k<<<grid, thr, smem, st>>>(y, zg, zf, g, J, (int)W, fd.pl, (const C*)fd.tw);
    return cudaGetLastError();
}

// =====================================================================================
// fft_grad_window: V_j[xi][col] = sum_b sum_w conj(X'_{b,j,w}[xi][k]) ZF_b[xi][k + iM]
// with k + iM = (col + a w) mod K0 (phase e^{+2 pi i xi/d} when it wraps);  grid (col-blocks, J)
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) fft_grad_window_kernel(const cplx<T>* __restrict__ y,
                                                                      const cplx<T>* __restrict__ zf,
                                                                      cplx<T>* __restrict__ v, SepGeom g, int64_t J,
                                                                      int64_t B, int64_t Bper, int W, FftPlanDev pl,
                                                                      const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int TILE = (int)g.d * W;
    C* acc = s + 2 * TILE;
    const int64_t j = blockIdx.y;
    const int64_t col0 = (int64_t)blockIdx.x * W;
    const int nbc = (int)min((int64_t)W, g.K0 - col0);
    const int total = (int)g.d * nbc;
    const int64_t Nsep = g.d * g.q;
    const T scale = (T)1 / (T)g.d;
    for (int e = threadIdx.x; e < total; e += blockDim.x) acc[e] = mk((T)0, (T)0);
    // signals [b0, b1) of this CTA's batch group; group z's sums go to v + z J L
    const int64_t b0 = (int64_t)blockIdx.z * Bper, b1 = min(B, b0 + Bper);
    for (int64_t b = b0; b < b1; ++b) {
        const C* yb = y + ((b * J + j) * Nsep) * g.M;
        const C* zfb = zf + b * g.L;
        for (int64_t w = 0; w < g.q; ++w) {
            __syncthreads();
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                const int nu = e / nbc, cc = e % nbc;
                int64_t t = col0 + cc + g.a * w;
                if (t >= g.K0) t -= g.K0;
                s[nu * W + cc] = yb[(w + g.q * nu) * g.M + (t % g.M)];
            }
            __syncthreads();
            const C* r = fft_tile<-1, true>(s, s + TILE, pl, nbc, W, 1, tw);
            for (int e = threadIdx.x; e < total; e += blockDim.x) {
                const int xi = e / nbc, cc = e % nbc;
                int64_t t = col0 + cc + g.a * w;
                const bool wrap = t >= g.K0;
                if (wrap) t -= g.K0;
                C u = cmulc(zfb[xi * g.K0 + t], cscale(r[xi * W + cc], scale));   // ZF * conj(X')
                if (wrap) u = cmulc(u, __ldg(tw + xi));
                acc[e] = cadd(acc[e], u);
            }
        }
    }
    __syncthreads();
    C* vj = v + ((int64_t)blockIdx.z * J + j) * g.L;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int xi = e / nbc, cc = e % nbc;
        vj[xi * g.K0 + col0 + cc] = acc[e];
    }
}

// v[e] = sum over the batch groups z of part[z n + e] (fixed order: deterministic)
template <typename T>
__global__ void sum_groups_kernel(const cplx<T>* __restrict__ part, cplx<T>* __restrict__ v, int64_t n, int groups) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        cplx<T> s = part[e];
        for (int z = 1; z < groups; ++z) s = cadd(s, part[z * n + e]);
        v[e] = s;
    }
}

int64_t fft_grad_window_groups(const SepGeom& g, int64_t J, int64_t B, size_t elem) {
    const int64_t elems = (int64_t)(kSmemBudget / elem);
    const int64_t W = std::min<int64_t>({elems / (3 * g.d), 16, g.K0});
    if (W < 1) return 1;
    const int64_t ctas = (g.K0 + W - 1) / W * J;
    // about eight CTAs per SM of a 152-SM device
    return std::max<int64_t>(1, std::min<int64_t>(B, (1216 + ctas - 1) / ctas));
}

template <typename T>
cudaError_t launch_fft_grad_window(const cplx<T>* y, const cplx<T>* zf, int64_t J, cplx<T>* v, cplx<T>* part,
                                   const SepGeom& g, const FftRef& fd, int64_t B, cudaStream_t st) {
    using C = cplx<T>;
    const int64_t elems = (int64_t)(kSmemBudget / sizeof(C));
    const int64_t W = std::min<int64_t>({elems / (3 * g.d), 16, g.K0});
    if (W < 1) return cudaErrorInvalidValue;
    const int64_t groups = part ? fft_grad_window_groups(g, J, B, sizeof(C)) : 1;
    const int64_t Bper = (B + groups - 1) / groups;
    const int64_t used = (B + Bper - 1) / Bper;               // groups that hold signals
    const int thr = threads_for(g.d * W);
    const size_t smem = sizeof(C) * (size_t)g.d * W * 3;
    auto k = fft_grad_window_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((g.K0 + W - 1) / W), (unsigned)J, (unsigned)used);
    k<<<grid, thr, smem, st>>>(y, zf, used > 1 ? part : v, g, J, B, Bper, (int)W, fd.pl, (const C*)fd.tw);
    e = cudaGetLastError();
    if (e != cudaSuccess || used <= 1) return e;
    const int64_t n = J * g.L;
    sum_groups_kernel<T><<<(unsigned)std::min<int64_t>((n + 255) / 256, 4096), 256, 0, st>>>(part, v, n, (int)used);
    return cudaGetLastError();
}

// =====================================================================================
// zak_inv (adjoint of zak_fwd): unnormalised inverse DFT over xi per column, post-op
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) zak_inv_kernel(const cplx<T>* __restrict__ zf, int64_t zbs,
                                                              void* __restrict__ dst, int dst_real, int64_t dbs,
                                                              int64_t d, int64_t K0, int W, FftPlanDev pl,
                                                              const cplx<T>* __restrict__ tw,
                                                              ChirpParams<cplx<T>> post, T scale) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int64_t b = blockIdx.y;
    const int64_t col0 = (int64_t)blockIdx.x * W;
    const int nbc = (int)min((int64_t)W, K0 - col0);
    const int total = (int)d * nbc;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = e / nbc, cc = e % nbc;
        s[i * W + cc] = zf[b * zbs + i * K0 + col0 + cc];
    }
    __syncthreads();
    const C* r = fft_tile<+1, true>(s, s + (int)d * W, pl, nbc, W, 1, tw);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = e / nbc, cc = e % nbc;
        const int64_t l = col0 + cc + K0 * i;
        C x = cscale(r[i * W + cc], scale);
        if (post.mode == PRE_CHIRP) x = cmul(x, chirp_factor(post, l));
        store_any(dst, dst_real, b * dbs + l, x);
    }
}

template <typename T>
cudaError_t launch_zak_inv(const cplx<T>* zf, int64_t zbs, void* dst, int dst_real, int64_t dbs, int64_t L, int64_t d,
                           const FftRef& fd, const ChirpParams<cplx<T>>& post, T scale, int64_t B, cudaStream_t st) {
    {
        cudaError_t e = p2_zak_inv<T>(zf, zbs, dst, dst_real, dbs, d, L / d, fd.tw, post, scale, B, st);
        if (e != cudaErrorNotSupported) return e;
        e = mr_zak_inv<T>(zf, zbs, dst, dst_real, dbs, d, L / d, fd.tw, post, scale, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    using C = cplx<T>;
    const int64_t K0 = L / d;
    const int64_t cap = tile_cap<T>();
    if (d > cap) return cudaErrorInvalidValue;
    // columns per CTA: a tile of about 48 KB (two buffers), so that several CTAs share an SM
    const int W = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)(24 * 1024 / sizeof(C)) / d, 16, K0}));
    const int thr = threads_for(d * W);
    const size_t smem = 2 * sizeof(C) * (size_t)d * W;
    auto k = zak_inv_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((K0 + W - 1) / W), (unsigned)B);
    k<<<grid, thr, smem, st>>>(zf, zbs, dst, dst_real, dbs, d, K0, W, fd.pl, (const C*)fd.tw, post, scale);
    return cudaGetLastError();
}

// =====================================================================================
// four-step FFT of length L = L1 L2, x[n1 L2 + n2] -> X[k1 + L1 k2]
//   cols: DFT over n1 per column n2 (pre-op on load), twiddle exp(dir 2 pi i n2 k1 / L)
//   rows: DFT over n2 per row k1, post-op and transposed (coalesced in k1) store
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) fftL_cols_kernel(const void* __restrict__ src, int src_real,
                                                                cplx<T>* __restrict__ tmp, int64_t L1, int64_t L2,
                                                                int dir, int W, FftPlanDev pl,
                                                                const cplx<T>* __restrict__ tw,
                                                                ChirpParams<cplx<T>> pre, CisTable<cplx<T>> cisL) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int64_t L = L1 * L2;
    const int64_t b = blockIdx.y;
    const int64_t c0 = (int64_t)blockIdx.x * W;
    const int nbc = (int)min((int64_t)W, L2 - c0);
    const int total = (int)L1 * nbc;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int i = e / nbc, cc = e % nbc;
        const int64_t l = (int64_t)i * L2 + c0 + cc;
        C x = load_any<C>(src, src_real, b * L + l);
        if (pre.mode == PRE_CHIRP) x = cmul(x, chirp_factor(pre, l));
        s[i * W + cc] = x;
    }
    __syncthreads();
    const int TILE = (int)L1 * W;
    const C* r = dir < 0 ? fft_tile<-1, true>(s, s + TILE, pl, nbc, W, 1, tw)
                         : fft_tile<+1, true>(s, s + TILE, pl, nbc, W, 1, tw);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int k1 = e / nbc, cc = e % nbc;
        const int64_t n2 = c0 + cc;
        const int64_t ex = (n2 * k1) % L;
        const C w = cisL(dir < 0 ? -ex : ex);
        tmp[b * L + (int64_t)k1 * L2 + n2] = cmul(r[k1 * W + cc], w);
    }
}

template <typename T>
__global__ void __launch_bounds__(kThreadsBig) fftL_rows_kernel(const cplx<T>* __restrict__ tmp, void* __restrict__ dst,
                                                                int dst_real, int64_t L1, int64_t L2, int dir, int R,
                                                                FftPlanDev pl, const cplx<T>* __restrict__ tw,
                                                                ChirpParams<cplx<T>> post, T scale) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int64_t L = L1 * L2;
    const int n = (int)L2;
    const int pitch = n + 1;
    const int64_t b = blockIdx.y;
    const int64_t r0 = (int64_t)blockIdx.x * R;
    const int nr = (int)min((int64_t)R, L1 - r0);
    const int total = nr * n;
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int r = e / n, k = e % n;
        s[r * pitch + k] = tmp[b * L + (r0 + r) * L2 + k];
    }
    __syncthreads();
    const int TILE = R * pitch;
    const C* res = dir < 0 ? fft_tile<-1, false>(s, s + TILE, pl, nr, 1, pitch, tw)
                           : fft_tile<+1, false>(s, s + TILE, pl, nr, 1, pitch, tw);
    for (int e = threadIdx.x; e < total; e += blockDim.x) {
        const int r = e % nr, k2 = e / nr;
        const int64_t kk = r0 + r + L1 * (int64_t)k2;
        C x = cscale(res[r * pitch + k2], scale);
        if (post.mode == PRE_CHIRP) x = cmul(x, chirp_factor(post, kk));
        store_any(dst, dst_real, b * L + kk, x);
    }
}

template <typename T>
cudaError_t launch_fftL_cols(const void* src, int src_real, cplx<T>* tmp, int64_t L1, int64_t L2, int dir,
                             const FftRef& f1, const ChirpParams<cplx<T>>& pre, const CisTable<cplx<T>>& cisL,
                             int64_t B, cudaStream_t st) {
    {
        cudaError_t e = mr_fftL_cols<T>(src, src_real, tmp, L1, L2, dir, f1.tw, pre, cisL, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    using C = cplx<T>;
    const int64_t cap = tile_cap<T>();
    if (L1 > cap) return cudaErrorInvalidValue;
    const int W = (int)std::max<int64_t>(1, std::min<int64_t>({cap / L1, 16, L2}));
    const int thr = threads_for(L1 * W);
    const size_t smem = 2 * sizeof(C) * (size_t)L1 * W;
    auto k = fftL_cols_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((L2 + W - 1) / W), (unsigned)B);
    k<<<grid, thr, smem, st>>>(src, src_real, tmp, L1, L2, dir, W, f1.pl, (const C*)f1.tw, pre, cisL);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_fftL_rows(const cplx<T>* tmp, void* dst, int dst_real, int64_t L1, int64_t L2, int dir,
                             const FftRef& f2, const ChirpParams<cplx<T>>& post, T scale, int64_t B,
                             cudaStream_t st) {
    {
        cudaError_t e = mr_fftL_rows<T>(tmp, dst, dst_real, L1, L2, dir, f2.tw, post, scale, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    using C = cplx<T>;
    const int64_t cap = tile_cap<T>();
    if (L2 + 1 > cap) return cudaErrorInvalidValue;
    const int R = (int)std::max<int64_t>(1, std::min<int64_t>({cap / (L2 + 1), 16, L1}));
    const int thr = threads_for(L2 * R);
    const size_t smem = 2 * sizeof(C) * (size_t)(L2 + 1) * R;
    auto k = fftL_rows_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    dim3 grid((unsigned)((L1 + R - 1) / R), (unsigned)B);
    k<<<grid, thr, smem, st>>>(tmp, dst, dst_real, L1, L2, dir, R, f2.pl, (const C*)f2.tw, post, scale);
    return cudaGetLastError();
}

// =====================================================================================
// FFT self-test: rows of length n, contiguous
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) fft_rows_test_kernel(const cplx<T>* __restrict__ in,
                                                                    cplx<T>* __restrict__ out, int64_t rows, int R,
                                                                    int dir, FftPlanDev pl,
                                                                    const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* s = reinterpret_cast<C*>(smem_raw);
    const int n = pl.n, pitch = n + 1;
    const int64_t row0 = (int64_t)blockIdx.x * R;
    const int nr = (int)min((int64_t)R, rows - row0);
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) s[(e / n) * pitch + e % n] = in[row0 * n + e];
    __syncthreads();
    const int TILE = R * pitch;
    const C* res = dir < 0 ? fft_tile<-1, false>(s, s + TILE, pl, nr, 1, pitch, tw)
                           : fft_tile<+1, false>(s, s + TILE, pl, nr, 1, pitch, tw);
    for (int e = threadIdx.x; e < nr * n; e += blockDim.x) out[row0 * n + e] = res[(e / n) * pitch + e % n];
}

template <typename T>
cudaError_t launch_fft_rows_test(const cplx<T>* in, cplx<T>* out, const FftRef& f, int dir, int64_t rows,
                                 cudaStream_t st) {
    using C = cplx<T>;
    const int64_t n = f.pl.n;
    const int64_t cap = tile_cap<T>();
    if (n + 1 > cap) return cudaErrorInvalidValue;
    // rows per CTA: a tile of about 48 KB (two buffers), so that several CTAs share an SM
    const int R = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)(24 * 1024 / sizeof(C)) / (n + 1), 16));
    const int thr = threads_for(n * R);
    const size_t smem = 2 * sizeof(C) * (size_t)(n + 1) * R;
    auto k = fft_rows_test_kernel<T>;
    cudaError_t e = prep_smem(k, smem);
    if (e != cudaSuccess) return e;
    k<<<(unsigned)((rows + R - 1) / R), thr, smem, st>>>(in, out, rows, R, dir, f.pl, (const C*)f.tw);
    return cudaGetLastError();
}

// explicit instantiations
#define DGT_INST(T)                                                                                                   \
    template cudaError_t launch_zak_fwd<T>(const void*, int, int64_t, cplx<T>*, int64_t, int64_t, int64_t,            \
                                           const FftRef&, const ChirpParams<cplx<T>>&, int64_t, cudaStream_t);        \
    template cudaError_t launch_prod_ifft<T>(const cplx<T>*, const cplx<T>*, int64_t, cplx<T>*, const SepGeom&,       \
                                             const FftRef&, int64_t, cudaStream_t);                                   \
    template cudaError_t launch_fft_post<T>(const cplx<T>*, cplx<T>*, const SepGeom&, int64_t, const FftRef&,         \
                                            const PostParams<cplx<T>>&, int64_t, cudaStream_t);                       \
    template cudaError_t launch_pre_ifft<T>(const cplx<T>*, cplx<T>*, const SepGeom&, int64_t, const FftRef&,         \
                                            const PostParams<cplx<T>>&, int64_t, cudaStream_t);                       \
    template cudaError_t launch_fft_prod_adj<T>(const cplx<T>*, const cplx<T>*, int64_t, cplx<T>*, const SepGeom&,    \
                                                const FftRef&, int64_t, unsigned int*, cudaStream_t);                 \
    template cudaError_t launch_fft_grad_window<T>(const cplx<T>*, const cplx<T>*, int64_t, cplx<T>*, cplx<T>*,       \
                                                   const SepGeom&, const FftRef&, int64_t, cudaStream_t);             \
    template cudaError_t launch_zak_inv<T>(const cplx<T>*, int64_t, void*, int, int64_t, int64_t, int64_t,            \
                                           const FftRef&, const ChirpParams<cplx<T>>&, T, int64_t, cudaStream_t);     \
    template cudaError_t launch_fftL_cols<T>(const void*, int, cplx<T>*, int64_t, int64_t, int, const FftRef&,        \
                                             const ChirpParams<cplx<T>>&, const CisTable<cplx<T>>&, int64_t,          \
                                             cudaStream_t);                                                           \
    template cudaError_t launch_fftL_rows<T>(const cplx<T>*, void*, int, int64_t, int64_t, int, const FftRef&,        \
                                             const ChirpParams<cplx<T>>&, T, int64_t, cudaStream_t);                  \
    template cudaError_t launch_fft_rows_test<T>(const cplx<T>*, cplx<T>*, const FftRef&, int, int64_t, cudaStream_t);

DGT_INST(float)
DGT_INST(double)

}  // namespace dgt
