// FIR (weighted overlap-add) path, window set-up, Gram blocks of the dual / tight windows,
// the window-gradient combination and the log-magnitude loss.
#include "engine.h"
#include "kcommon.cuh"

#include <algorithm>
#include <map>
#include <mutex>

namespace dgt {

template <typename C> __device__ __forceinline__ C load_any2(const void* p, int is_real, int64_t i) {
    using R = typename RealOf<C>::type;
    if (is_real) return mk(reinterpret_cast<const R*>(p)[i], (R)0);
    return reinterpret_cast<const C*>(p)[i];
}

// Transform nr rows (pitch elements apart) in groups of `group` rows, each group ping-ponged
// with the spare buffer of `group` rows; results end in place.  Ends synchronised.
template <int DIR, typename C>
__device__ void fft_rows_grouped(C* rows, C* spare, int nr, int group, int pitch, const FftPlanDev& pl,
                                 const C* __restrict__ tw) {
    for (int g0 = 0; g0 < nr; g0 += group) {
        const int ng = min(group, nr - g0);
        C* a = rows + (size_t)g0 * pitch;
        const C* res = fft_tile<DIR, false>(a, spare, pl, ng, 1, pitch, tw);
        if (res != a) {
            for (int e = threadIdx.x; e < ng * pitch; e += blockDim.x) a[e] = res[e];
            __syncthreads();
        }
    }
}

static size_t g_smem_optin2 = 0;
template <typename K> static cudaError_t prep_smem2(K kernel, size_t bytes) {
    if (g_smem_optin2 == 0) {
        int dev = 0, v = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
        g_smem_optin2 = (size_t)v;
    }
    if (bytes > g_smem_optin2) return cudaErrorInvalidValue;
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    return cudaSuccess;
}

// =====================================================================================
// FIR analysis: for a chunk of `cols` time positions n of one signal,
//   h_n(k) = sum_{x : (a n + x) mod M = k} f(a n + x) conj(g(x)) e^{-2 pi i (a n + x) w(n) / M}
//   c(., n) = FFT_M(h_n)          (eq. DGT folded modulo M; cost of eq. rect-flops-FIR)
// x runs over the window support [-center, Lg - center).  grid (chunks, B)
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) fir_analysis_kernel(const void* __restrict__ f, int f_real,
                                                                   cplx<T>* __restrict__ c, FirParams<cplx<T>> fp,
                                                                   FftPlanDev pl, const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = pl.n, pitch = M + 1;
    const int64_t b = blockIdx.y;
    const int64_t n0 = (int64_t)blockIdx.x * fp.cols;
    const int nc = (int)min(fp.cols, fp.N - n0);
    const int64_t S = fp.a * (nc - 1) + fp.Lg;                // segment length
    C* rows = reinterpret_cast<C*>(smem_raw);
    C* spare = rows + (size_t)fp.cols * pitch;
    C* seg = spare + (size_t)fp.group * pitch;
    const int64_t lstart = fp.a * n0 - fp.center;
    for (int64_t t = threadIdx.x; t < S; t += blockDim.x) {
        const int64_t l = posmod(lstart + t, fp.L);
        seg[t] = load_any2<C>(f, f_real, b * fp.L + l);
    }
    __syncthreads();
    const int64_t LM = fp.lam2 * fp.M;
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int r = e / M, k = e % M;
        const int64_t n = n0 + r;
        const int64_t ln = fp.a * n - fp.center;              // time of tap 0
        const int64_t wn = (n * fp.lam1) % fp.lam2;
        int64_t t = posmod((int64_t)k - ln, fp.M);            // first tap folding onto k
        C h = mk((T)0, (T)0);
        for (; t < fp.Lg; t += fp.M) {
            const int64_t l = posmod(ln + t, fp.L);
            C v = cmulc(seg[fp.a * r + t], __ldg(fp.taps + t));
            if (wn) v = cmul(v, fp.cisLM(-(int64_t)mulmod((uint64_t)(l % LM), (uint64_t)wn, (uint64_t)LM)));
            h = cadd(h, v);
        }
        rows[r * pitch + k] = h;
    }
    __syncthreads();
    fft_rows_grouped<-1>(rows, spare, nc, (int)fp.group, pitch, pl, tw);
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int r = e / M, m = e % M;
        c[(b * fp.N + n0 + r) * fp.M + m] = rows[r * pitch + m];
    }
}

template <typename C> int64_t fir_seam_elems(const FirParams<C>& fp) {
    const int64_t ov = std::max<int64_t>(0, fp.Lg - fp.a);
    return (fp.N / fp.cols) * 2 * ov;
}
template int64_t fir_seam_elems<float2>(const FirParams<float2>&);
template int64_t fir_seam_elems<double2>(const FirParams<double2>&);

template <typename T>
cudaError_t launch_fir_analysis(const void* f, int f_real, cplx<T>* c, const FirParams<cplx<T>>& fp,
                                const FftRef& fm, int64_t B, cudaStream_t st) {
    using C = cplx<T>;
    {
        const cudaError_t e = p2_fir_analysis<T>(f, f_real, c, fp, fm.tw, B, st);
        if (e != cudaErrorNotSupported) return e;
    }
    if (fp.half) return cudaErrorNotSupported;       // half-channel output: power-of-two kernels only
    const int64_t S = fp.a * (fp.cols - 1) + fp.Lg;
    const size_t smem = sizeof(C) * ((size_t)(fp.cols + fp.group) * (fp.M + 1) + S);
    if (smem > kSmemBudget) return cudaErrorInvalidValue;
    auto k = fir_analysis_kernel<T>;
    cudaError_t e = prep_smem2(k, smem);
    if (e != cudaSuccess) return e;
    const int thr = threads_for(fp.cols * fp.M);
    dim3 grid((unsigned)((fp.N + fp.cols - 1) / fp.cols), (unsigned)B);
    k<<<grid, thr, smem, st>>>(f, f_real, c, fp, fm.pl, (const C*)fm.tw);
    return cudaGetLastError();
}

// =====================================================================================
// FIR synthesis (adjoint): per chunk of `cols` columns, unnormalised inverse FFT_M of each
// column, then for every sample of the chunk's segment gather
//   f(l) = sum_n gamma(l - a n) e^{+2 pi i l w(n)/M} h_n(l mod M)
// Samples reached only by this chunk's columns are stored; the two seams of Lg - a samples
// shared with the neighbouring chunks go to a seam buffer and are summed by fir_seams.
// Requires N % cols == 0 and a * cols >= Lg - a (host-checked).
// =====================================================================================
template <typename T>
__global__ void __launch_bounds__(kThreadsBig) fir_synthesis_kernel(const cplx<T>* __restrict__ c, void* __restrict__ f,
                                                                    int f_real, cplx<T>* __restrict__ seams,
                                                                    FirParams<cplx<T>> fp, FftPlanDev pl,
                                                                    const cplx<T>* __restrict__ tw) {
    using C = cplx<T>;
    using R = T;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int M = pl.n, pitch = M + 1;
    const int64_t b = blockIdx.y;
    const int64_t chunk = blockIdx.x;
    const int64_t nchunks = gridDim.x;
    const int64_t n0 = chunk * fp.cols;
    const int nc = (int)fp.cols;
    C* rows = reinterpret_cast<C*>(smem_raw);
    C* spare = rows + (size_t)fp.cols * pitch;
    for (int e = threadIdx.x; e < nc * M; e += blockDim.x) {
        const int r = e / M, m = e % M;
        rows[r * pitch + m] = c[(b * fp.N + n0 + r) * fp.M + m];
    }
    __syncthreads();
    fft_rows_grouped<+1>(rows, spare, nc, (int)fp.group, pitch, pl, tw);
    const int64_t S = fp.a * (nc - 1) + fp.Lg;
    const int64_t ov = fp.Lg > fp.a ? fp.Lg - fp.a : 0;
    const int64_t lstart = fp.a * n0 - fp.center;
    const int64_t LM = fp.lam2 * fp.M;
    const int64_t soff = (b * nchunks + chunk) * 2 * ov;
    C* seamL = f_real ? reinterpret_cast<C*>(reinterpret_cast<R*>(seams) + soff) : seams + soff;
    for (int64_t t = threadIdx.x; t < S; t += blockDim.x) {
        const int64_t l = posmod(lstart + t, fp.L);
        const int64_t km = l % fp.M;
        C acc = mk((T)0, (T)0);
        // columns r with 0 <= t - a r < Lg
        int64_t rlo = t - fp.Lg + 1 <= 0 ? 0 : (t - fp.Lg + fp.a) / fp.a;
        int64_t rhi = min((int64_t)nc - 1, t / fp.a);
        for (int64_t r = rlo; r <= rhi; ++r) {
            const int64_t tap = t - fp.a * r;
            const int64_t n = n0 + r;
            const int64_t wn = (n * fp.lam1) % fp.lam2;
            C v = cmul(rows[r * pitch + km], __ldg(fp.taps + tap));
            if (wn) v = cmul(v, fp.cisLM((int64_t)mulmod((uint64_t)(l % LM), (uint64_t)wn, (uint64_t)LM)));
            acc = cadd(acc, v);
        }
        if (t < ov || t >= S - ov) {
            const int64_t si = t < ov ? t : ov + t - (S - ov);      // seams of a real output are stored real
            if (f_real) reinterpret_cast<R*>(seamL)[si] = acc.x;
            else seamL[si] = acc;
        } else {
            if (f_real) reinterpret_cast<R*>(f)[b * fp.L + l] = acc.x;
            else reinterpret_cast<C*>(f)[b * fp.L + l] = acc;
        }
    }
}

template <typename T>
__global__ void fir_seams_kernel(const cplx<T>* __restrict__ seams, void* __restrict__ f, int f_real,
                                 FirParams<cplx<T>> fp, int64_t nchunks, int64_t B) {
    using C = cplx<T>;
    const int64_t ov = fp.Lg - fp.a;
    const int64_t total = B * nchunks * ov;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = e % ov;
        const int64_t chunk = (e / ov) % nchunks;
        const int64_t b = e / (ov * nchunks);
        const int64_t nxt = (chunk + 1) % nchunks;
        const int64_t ir = (b * nchunks + chunk) * 2 * ov + ov + t, il = (b * nchunks + nxt) * 2 * ov + t;
        const int64_t l = posmod(fp.a * (chunk + 1) * fp.cols - fp.center + t, fp.L);
        if (f_real) {                                       // real seams for a real output
            const T* sr = reinterpret_cast<const T*>(seams);
            reinterpret_cast<T*>(f)[b * fp.L + l] = sr[ir] + sr[il];
        } else {
            reinterpret_cast<C*>(f)[b * fp.L + l] = cadd(seams[ir], seams[il]);
        }
    }
}

template <typename T>
cudaError_t launch_fir_synthesis(const cplx<T>* c, void* f, int f_real, cplx<T>* seams, const FirParams<cplx<T>>& fp,
                                 const FftRef& fm, int64_t B, cudaStream_t st) {
    using C = cplx<T>;
    if (fp.N % fp.cols) return cudaErrorInvalidValue;
    if (fp.a * fp.cols < fp.Lg - fp.a) return cudaErrorInvalidValue;
    const int64_t nchunks = fp.N / fp.cols;
    cudaError_t e = p2_fir_synthesis<T>(c, f, f_real, seams, fp, fm.tw, B, st);
    if (e == cudaErrorNotSupported && fp.half) return e;  // half-channel input: power-of-two kernels only
    if (e == cudaErrorNotSupported) {
        const size_t smem = sizeof(C) * ((size_t)(fp.cols + fp.group) * (fp.M + 1));
        if (smem > kSmemBudget) return cudaErrorInvalidValue;
        auto k = fir_synthesis_kernel<T>;
        e = prep_smem2(k, smem);
        if (e != cudaSuccess) return e;
        const int thr = threads_for(fp.cols * fp.M);
        dim3 grid((unsigned)nchunks, (unsigned)B);
        k<<<grid, thr, smem, st>>>(c, f, f_real, seams, fp, fm.pl, (const C*)fm.tw);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return e;
    if (fp.Lg > fp.a) {
        const int64_t total = B * nchunks * (fp.Lg - fp.a);
        const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 16);
        fir_seams_kernel<T><<<blocks, 256, 0, st>>>(seams, f, f_real, fp, nchunks, B);
        e = cudaGetLastError();
    }
    return e;
}

// =====================================================================================
// window set-up helpers
// =====================================================================================
// g_j(l) = exp(2 pi i sigma_j l / L) g(l - j a)   (Prop. mw_frop: g_j = M_{sigma_j} T_{ja} g)
template <typename T>
__global__ void coset_windows_kernel(const cplx<T>* __restrict__ g, cplx<T>* __restrict__ gj, int64_t L, int64_t a,
                                     int64_t J, const int64_t* __restrict__ sigma, CisTable<cplx<T>> cisL) {
    const int64_t total = J * L;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / L, l = e % L;
        const int64_t src = posmod(l - j * a, L);
        const int64_t ex = (int64_t)mulmod((uint64_t)l, (uint64_t)sigma[j], (uint64_t)L);
        gj[e] = cmul(g[src], cisL(ex));
    }
}

template <typename T>
cudaError_t launch_coset_windows(const cplx<T>* g, cplx<T>* gj, int64_t L, int64_t a, int64_t J, const int64_t* sigma,
                                 const CisTable<cplx<T>>& cisL, cudaStream_t st) {
    const int64_t total = J * L;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32);
    coset_windows_kernel<T><<<blocks, 256, 0, st>>>(g, gj, L, a, J, sigma, cisL);
    return cudaGetLastError();
}

// tab[l] = pchirp(L, s)(l), l < L (Algorithm 1's chirps), from the exact exponent: the table the
// per-sample chirp_factor reads instead of three reductions modulo 2L and a two-level lookup
template <typename T>
__global__ void chirp_table_kernel(ChirpParams<cplx<T>> cp, cplx<T>* __restrict__ tab) {
    for (int64_t l = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; l < cp.L; l += (int64_t)gridDim.x * blockDim.x)
        tab[l] = chirp_exact(cp, l);
}

template <typename T>
cudaError_t launch_chirp_table(const ChirpParams<cplx<T>>& cp, cplx<T>* tab, cudaStream_t st) {
    ChirpParams<cplx<T>> c = cp;
    c.conj = 0;
    c.tab = nullptr;
    const unsigned blocks = (unsigned)std::min<int64_t>((cp.L + 255) / 256, 152 * 32);
    chirp_table_kernel<T><<<blocks, 256, 0, st>>>(c, tab);
    return cudaGetLastError();
}

template <typename Tin, typename Tout>
__global__ void convert_kernel(const void* __restrict__ in, int in_real, cplx<Tout>* __restrict__ out, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        if (in_real) out[e] = mk((Tout)reinterpret_cast<const Tin*>(in)[e], (Tout)0);
        else {
            const cplx<Tin> v = reinterpret_cast<const cplx<Tin>*>(in)[e];
            out[e] = mk((Tout)v.x, (Tout)v.y);
        }
    }
}

template <typename Tin, typename Tout>
cudaError_t launch_convert(const void* in, int in_real, cplx<Tout>* out, int64_t n, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::min<int64_t>((n + 255) / 256, 152 * 32);
    convert_kernel<Tin, Tout><<<blocks, 256, 0, st>>>(in, in_real, out, n);
    return cudaGetLastError();
}

// grad_g(y) = sum_j exp(-2 pi i sigma_j (y + j a) / L) W_j(y + j a): adjoint of g -> g_j
template <typename T>
__global__ void grad_combine_kernel(const cplx<T>* __restrict__ wj, void* __restrict__ grad, int grad_real, int64_t L,
                                    int64_t a, int64_t J, const int64_t* __restrict__ sigma, CisTable<cplx<T>> cisL) {
    using C = cplx<T>;
    for (int64_t y = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; y < L; y += (int64_t)gridDim.x * blockDim.x) {
        C acc = mk((T)0, (T)0);
        for (int64_t j = 0; j < J; ++j) {
            const int64_t x = (y + j * a) % L;
            const int64_t ex = (int64_t)mulmod((uint64_t)x, (uint64_t)sigma[j], (uint64_t)L);
            acc = cadd(acc, cmul(wj[j * L + x], cisL(-ex)));
        }
        if (grad_real) reinterpret_cast<T*>(grad)[y] = acc.x;
        else reinterpret_cast<C*>(grad)[y] = acc;
    }
}

template <typename T>
cudaError_t launch_grad_window_combine(const cplx<T>* wj, void* grad, int grad_real, int64_t L, int64_t a, int64_t J,
                                       const int64_t* sigma, const CisTable<cplx<T>>& cisL, cudaStream_t st) {
    const unsigned blocks = (unsigned)std::min<int64_t>((L + 255) / 256, 152 * 32);
    grad_combine_kernel<T><<<blocks, 256, 0, st>>>(wj, grad, grad_real, L, a, J, sigma, cisL);
    return cudaGetLastError();
}

// u = 2 c / (|c|^2 + eps) (gradient of sum log(|c|^2 + eps) in the d/dRe + i d/dIm
// convention) and per-block partial sums of log(|c|^2 + eps), for B signals of n coefficients.
template <typename T>
__global__ void logmag_kernel(const cplx<T>* __restrict__ c, cplx<T>* __restrict__ u, double* __restrict__ partial,
                              int64_t n, T eps) {
    __shared__ double red[256];
    const int64_t b = blockIdx.y;
    // float: single-precision logarithms summed with a compensated (Kahan) float sum per thread,
    // then a float64 tree over the CTA; float64: the float64 logarithm and sum
    T acc = 0, comp = 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const cplx<T> v = c[b * n + e];
        const T m2 = v.x * v.x + v.y * v.y + eps;
        const T y = log(m2) - comp;
        const T s = acc + y;
        comp = (s - acc) - y;
        acc = s;
        if (u) {
            T inv;
            if constexpr (sizeof(T) == 4) inv = __fdividef(2.f, m2);
            else inv = (T)2 / m2;
            u[b * n + e] = cscale(v, inv);
        }
    }
    red[threadIdx.x] = (double)acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[b * gridDim.x + blockIdx.x] = red[0];
}

// loss_b = sum of the P partial sums of signal b (float64)
__global__ void logmag_finish_kernel(const double* __restrict__ partial, double* __restrict__ loss, int P) {
    __shared__ double red[64];
    const int64_t b = blockIdx.x;
    red[threadIdx.x] = threadIdx.x < P ? partial[b * P + threadIdx.x] : 0.0;
    __syncthreads();
    for (int s = 32; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) loss[b] = red[0];
}

template <typename T>
cudaError_t launch_logmag(const cplx<T>* c, cplx<T>* u, double* partial, double* loss, int64_t n, T eps, int64_t B,
                          cudaStream_t st) {
    constexpr int P = 64;
    logmag_kernel<T><<<dim3(P, (unsigned)B), 256, 0, st>>>(c, u, partial, n, eps);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    logmag_finish_kernel<<<(unsigned)B, 64, 0, st>>>(partial, loss, P);
    return cudaGetLastError();
}

// =====================================================================================
// Gram blocks (float64).  For the separable lattice (at, M) of the coset decomposition and
// every (xi, k < M):  Phi_j[i][w] = ZG~_j[xi][k + iM - at w] (i < p, w < q),
// G = M sum_j Phi_j Phi_j^H (p x p), right-hand side ZG_0[xi][k + iM].
// dual:  Zgamma = G^{-1} rhs ;  tight: Zgamma = G^{-1/2} rhs.
// =====================================================================================
constexpr int kPMax = 8;

__device__ void herm_jacobi(double2 (&A)[kPMax][kPMax], double2 (&V)[kPMax][kPMax], int p) {
    // cyclic Jacobi for a Hermitian p x p matrix: A <- V^H A V diagonal, V unitary
    for (int i = 0; i < p; ++i)
        for (int j = 0; j < p; ++j) V[i][j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
    for (int sweep = 0; sweep < 30; ++sweep) {
        double off = 0, tot = 0;
        for (int i = 0; i < p; ++i)
            for (int j = 0; j < p; ++j) {
                const double m = A[i][j].x * A[i][j].x + A[i][j].y * A[i][j].y;
                tot += m;
                if (i != j) off += m;
            }
        if (off <= 1e-30 * tot) break;
        for (int pp = 0; pp < p - 1; ++pp)
            for (int q = pp + 1; q < p; ++q) {
                const double2 apq = A[pp][q];
                const double mag = sqrt(apq.x * apq.x + apq.y * apq.y);
                if (mag < 1e-300) continue;
                const double2 ph = make_double2(apq.x / mag, apq.y / mag);     // e^{i phi}
                const double app = A[pp][pp].x, aqq = A[q][q].x;
                const double theta = 0.5 * atan2(2 * mag, aqq - app);
                const double cs = cos(theta), sn = sin(theta);
                // rotation acting on columns pp, q:  [c, s e^{i phi}; -s e^{-i phi}, c]
                for (int k = 0; k < p; ++k) {
                    const double2 akp = A[k][pp], akq = A[k][q];
                    // A[:,pp] = c akp - s e^{-i phi} akq ; A[:,q] = s e^{i phi} akp + c akq
                    const double2 t1 = cmulc(akq, ph);
                    const double2 t2 = cmul(akp, ph);
                    A[k][pp] = make_double2(cs * akp.x - sn * t1.x, cs * akp.y - sn * t1.y);
                    A[k][q] = make_double2(sn * t2.x + cs * akq.x, sn * t2.y + cs * akq.y);
                    const double2 vkp = V[k][pp], vkq = V[k][q];
                    const double2 u1 = cmulc(vkq, ph);
                    const double2 u2 = cmul(vkp, ph);
                    V[k][pp] = make_double2(cs * vkp.x - sn * u1.x, cs * vkp.y - sn * u1.y);
                    V[k][q] = make_double2(sn * u2.x + cs * vkq.x, sn * u2.y + cs * vkq.y);
                }
                for (int k = 0; k < p; ++k) {
                    const double2 apk = A[pp][k], aqk = A[q][k];
                    // rows: A[pp,:] = c apk - s e^{i phi} aqk ; A[q,:] = s e^{-i phi} apk + c aqk
                    const double2 t1 = cmul(aqk, ph);
                    const double2 t2 = cmulc(apk, ph);
                    A[pp][k] = make_double2(cs * apk.x - sn * t1.x, cs * apk.y - sn * t1.y);
                    A[q][k] = make_double2(sn * t2.x + cs * aqk.x, sn * t2.y + cs * aqk.y);
                }
            }
    }
}

__global__ void gram_solve_kernel(const double2* __restrict__ zg, int64_t J, double2* __restrict__ zout, SepGeom g,
                                  int tight, int* __restrict__ status) {
    const int64_t total = g.d * g.M;
    const double2* ZG0 = zg;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t xi = e / g.M, k = e % g.M;
        const int p = (int)g.p;
        const double2 unwrap = make_double2(cospi(-2.0 * (double)xi / (double)g.d), sinpi(-2.0 * (double)xi / (double)g.d));
        double2 G[kPMax][kPMax];
        for (int i = 0; i < p; ++i)
            for (int i2 = 0; i2 < p; ++i2) G[i][i2] = make_double2(0, 0);
        for (int64_t j = 0; j < J; ++j) {
            const double2* Z = zg + j * g.L;
            for (int64_t w = 0; w < g.q; ++w) {
                double2 phi[kPMax];
                for (int i = 0; i < p; ++i) {
                    int64_t col = k + i * g.M - g.a * w;
                    const bool wrap = col < 0;
                    if (wrap) col += g.K0;
                    double2 v = Z[xi * g.K0 + col];
                    if (wrap) v = cmul(v, unwrap);
                    phi[i] = v;
                }
                for (int i = 0; i < p; ++i)
                    for (int i2 = 0; i2 < p; ++i2) G[i][i2] = cadd(G[i][i2], cmulc(phi[i], phi[i2]));
            }
        }
        const double Md = (double)g.M;
        double2 rhs[kPMax], x[kPMax];
        for (int i = 0; i < p; ++i) rhs[i] = ZG0[xi * g.K0 + k + i * g.M];
        for (int i = 0; i < p; ++i)
            for (int i2 = 0; i2 < p; ++i2) G[i][i2] = cscale(G[i][i2], Md);
        if (p == 1) {
            const double gv = G[0][0].x;
            if (!(gv > 0)) atomicExch(status, 1);
            x[0] = cscale(rhs[0], tight ? 1.0 / sqrt(gv) : 1.0 / gv);
        } else if (!tight) {
            // Gaussian elimination with partial pivoting
            double2 A[kPMax][kPMax];
            for (int i = 0; i < p; ++i) {
                for (int i2 = 0; i2 < p; ++i2) A[i][i2] = G[i][i2];
                x[i] = rhs[i];
            }
            double dmax = 0;
            for (int i = 0; i < p; ++i) dmax = fmax(dmax, A[i][i].x);
            for (int col = 0; col < p; ++col) {
                int piv = col;
                double best = 0;
                for (int r = col; r < p; ++r) {
                    const double m = hypot(A[r][col].x, A[r][col].y);
                    if (m > best) { best = m; piv = r; }
                }
                if (!(best > 1e-14 * dmax)) { atomicExch(status, 1); best = 1; }
                if (piv != col) {
                    for (int i2 = 0; i2 < p; ++i2) { double2 t = A[col][i2]; A[col][i2] = A[piv][i2]; A[piv][i2] = t; }
                    double2 t = x[col]; x[col] = x[piv]; x[piv] = t;
                }
                const double2 pv = A[col][col];
                const double den = pv.x * pv.x + pv.y * pv.y;
                const double2 inv = den > 0 ? make_double2(pv.x / den, -pv.y / den) : make_double2(0, 0);
                for (int r = 0; r < p; ++r) {
                    if (r == col) continue;
                    const double2 fct = cmul(A[r][col], inv);
                    for (int i2 = col; i2 < p; ++i2) A[r][i2] = csub(A[r][i2], cmul(fct, A[col][i2]));
                    x[r] = csub(x[r], cmul(fct, x[col]));
                }
            }
            for (int i = 0; i < p; ++i) {
                const double2 pv = A[i][i];
                const double den = pv.x * pv.x + pv.y * pv.y;
                x[i] = den > 0 ? cmul(x[i], make_double2(pv.x / den, -pv.y / den)) : make_double2(0, 0);
            }
        } else {
            double2 V[kPMax][kPMax];
            herm_jacobi(G, V, p);
            double lmax = 0;
            for (int i = 0; i < p; ++i) lmax = fmax(lmax, G[i][i].x);
            double2 tmp[kPMax];
            for (int i = 0; i < p; ++i) {      // tmp = V^H rhs / sqrt(lambda)
                double2 s = make_double2(0, 0);
                for (int r = 0; r < p; ++r) s = cadd(s, cmulc(rhs[r], V[r][i]));
                const double lam = G[i][i].x;
                if (!(lam > 1e-14 * lmax)) { atomicExch(status, 1); }
                tmp[i] = lam > 0 ? cscale(s, 1.0 / sqrt(lam)) : make_double2(0, 0);
            }
            for (int r = 0; r < p; ++r) {
                double2 s = make_double2(0, 0);
                for (int i = 0; i < p; ++i) s = cadd(s, cmul(V[r][i], tmp[i]));
                x[r] = s;
            }
        }
        for (int i = 0; i < p; ++i) zout[xi * g.K0 + k + i * g.M] = x[i];
    }
}

cudaError_t launch_gram_solve(const double2* zg, int64_t J, double2* zout, const SepGeom& g, int tight, int* status,
                              cudaStream_t st) {
    if (g.p > kPMax) return cudaErrorInvalidValue;
    const int64_t total = g.d * g.M;
    const unsigned blocks = (unsigned)std::min<int64_t>((total + 127) / 128, 152 * 16);
    gram_solve_kernel<<<blocks, 128, 0, st>>>(zg, J, zout, g, tight, status);
    return cudaGetLastError();
}

// gamma(x) = g(x) / (M sum_{x' = x mod a} |g(x')|^2)  (tight: square root of the denominator);
// exact when the window support is at most M long.
__global__ void fir_dual_kernel(const double2* __restrict__ taps, double2* __restrict__ out, int64_t Lg, int64_t a,
                                int64_t M, int tight, int* __restrict__ status) {
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < Lg; t += (int64_t)gridDim.x * blockDim.x) {
        double s = 0;
        for (int64_t u = t % a; u < Lg; u += a) s += taps[u].x * taps[u].x + taps[u].y * taps[u].y;
        s *= (double)M;
        if (!(s > 0)) {
            // a sample no window translate reaches: no frame
            atomicExch(status, 1);
            out[t] = make_double2(0, 0);
            continue;
        }
        out[t] = cscale(taps[t], tight ? 1.0 / sqrt(s) : 1.0 / s);
    }
}

cudaError_t launch_fir_dual(const double2* taps, double2* out, int64_t Lg, int64_t a, int64_t M, int tight, int* status,
                            cudaStream_t st) {
    fir_dual_kernel<<<(unsigned)std::min<int64_t>((Lg + 255) / 256, 1024), 256, 0, st>>>(taps, out, Lg, a, M, tight,
                                                                                         status);
    return cudaGetLastError();
}

// Modulated FIR taps out[wn][t] = conj(h(t)) exp(-2 pi i ((t wn) mod lam2 M) / (lam2 M)),
// computed in float64 from the exactly reduced integer phase, then rounded once to T.
template <typename T>
__global__ void fir_modtaps_kernel(const double2* __restrict__ h, cplx<T>* __restrict__ out, int64_t Lg, int64_t lam2,
                                   int64_t M) {
    const int64_t LM = lam2 * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < lam2 * Lg;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t wn = e / Lg, t = e - wn * Lg;
        const int64_t r = (t % LM) * wn % LM;
        double sn, cs;
        sincospi(2.0 * (double)r / (double)LM, &sn, &cs);
        const double2 v = cmulc(make_double2(cs, -sn), h[t]);
        out[e] = mk((T)v.x, (T)v.y);
    }
}

template <typename T>
cudaError_t launch_fir_modtaps(const double2* h, cplx<T>* out, int64_t Lg, int64_t lam2, int64_t M, cudaStream_t st) {
    const int64_t n = lam2 * Lg;
    fir_modtaps_kernel<T><<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, 0, st>>>(h, out, Lg, lam2, M);
    return cudaGetLastError();
}
template cudaError_t launch_fir_modtaps<float>(const double2*, float2*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_fir_modtaps<double>(const double2*, double2*, int64_t, int64_t, int64_t, cudaStream_t);

// =====================================================================================
// Blockwise (overlap-add) DGT: block buffers and the column map between the blocks' short
// transforms (length Lx, Nx = Lx / a columns) and the long one (N columns).  Block beta
// starts at sample beta Lb; its local column nu' stands for the global column
// (beta S + nu) mod N, S = Lb / a, nu = nu' for nu' <= nu_hi and nu' - Nx otherwise.
// =====================================================================================
template <typename E>
__global__ void ola_split_kernel(const E* __restrict__ f, E* __restrict__ x, OlaGeom og, int64_t B) {
    const int64_t total = B * og.Nb * og.Lx;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = e % og.Lx, bb = e / og.Lx;            // bb = b Nb + beta
        E v{};
        if (u < og.Lb) v = f[bb * og.Lb + u];                    // block beta of signal b is contiguous
        x[e] = v;
    }
}

template <typename E>
__global__ void ola_take_kernel(const E* __restrict__ y, E* __restrict__ f, OlaGeom og, int64_t B) {
    const int64_t total = B * og.Nb * og.Lb;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = e % og.Lb, bb = e / og.Lb;
        f[e] = y[bb * og.Lx + u];
    }
}

// c[b][n][m] = sum over the blocks whose columns include n, in increasing distance order
template <typename C>
__global__ void ola_add_kernel(const C* __restrict__ cx, C* __restrict__ c, OlaGeom og, int64_t B) {
    const int64_t total = B * og.N * og.M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e % og.M, r = e / og.M;
        const int64_t n = r % og.N, b = r / og.N;
        // the latest block that can reach n through a wrapped (negative) local column
        const int64_t top = (n + (og.Nx - og.nu_hi - 1)) / og.S;
        C acc{};
        for (int64_t k = 0; k < og.K; ++k) {
            int64_t beta = (top - k) % og.Nb;
            if (beta < 0) beta += og.Nb;
            int64_t delta = (n - beta * og.S) % og.N;
            if (delta < 0) delta += og.N;
            int64_t nu;
            if (delta <= og.nu_hi) nu = delta;
            else if (delta >= og.N - (og.Nx - og.nu_hi - 1)) nu = delta - og.N + og.Nx;
            else continue;
            const C v = cx[((b * og.Nb + beta) * og.Nx + nu) * og.M + m];
            acc.x += v.x;
            acc.y += v.y;
        }
        c[e] = acc;
    }
}

template <typename C>
__global__ void ola_gather_kernel(const C* __restrict__ c, C* __restrict__ cx, OlaGeom og, int64_t B) {
    const int64_t total = B * og.Nb * og.Nx * og.M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e % og.M, r = e / og.M;
        const int64_t nu = r % og.Nx, bb = r / og.Nx;
        const int64_t beta = bb % og.Nb, b = bb / og.Nb;
        int64_t n = (beta * og.S + (nu <= og.nu_hi ? nu : nu - og.Nx)) % og.N;
        if (n < 0) n += og.N;
        cx[e] = c[(b * og.N + n) * og.M + m];
    }
}

static unsigned ola_blocks(int64_t total) { return (unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32); }

template <typename T>
cudaError_t launch_ola_split(const void* f, int f_real, void* x, const OlaGeom& og, int64_t B, cudaStream_t st) {
    const int64_t total = B * og.Nb * og.Lx;
    if (f_real) ola_split_kernel<T><<<ola_blocks(total), 256, 0, st>>>((const T*)f, (T*)x, og, B);
    else ola_split_kernel<cplx<T>><<<ola_blocks(total), 256, 0, st>>>((const cplx<T>*)f, (cplx<T>*)x, og, B);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_ola_take(const void* y, int f_real, void* f, const OlaGeom& og, int64_t B, cudaStream_t st) {
    const int64_t total = B * og.Nb * og.Lb;
    if (f_real) ola_take_kernel<T><<<ola_blocks(total), 256, 0, st>>>((const T*)y, (T*)f, og, B);
    else ola_take_kernel<cplx<T>><<<ola_blocks(total), 256, 0, st>>>((const cplx<T>*)y, (cplx<T>*)f, og, B);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_ola_add(const cplx<T>* cx, cplx<T>* c, const OlaGeom& og, int64_t B, cudaStream_t st) {
    ola_add_kernel<cplx<T>><<<ola_blocks(B * og.N * og.M), 256, 0, st>>>(cx, c, og, B);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_ola_gather(const cplx<T>* c, cplx<T>* cx, const OlaGeom& og, int64_t B, cudaStream_t st) {
    ola_gather_kernel<cplx<T>><<<ola_blocks(B * og.Nb * og.Nx * og.M), 256, 0, st>>>(c, cx, og, B);
    return cudaGetLastError();
}
#define DGT_INST_OLA(T)                                                                                         \
    template cudaError_t launch_ola_split<T>(const void*, int, void*, const OlaGeom&, int64_t, cudaStream_t);   \
    template cudaError_t launch_ola_take<T>(const void*, int, void*, const OlaGeom&, int64_t, cudaStream_t);    \
    template cudaError_t launch_ola_add<T>(const cplx<T>*, cplx<T>*, const OlaGeom&, int64_t, cudaStream_t);   \
    template cudaError_t launch_ola_gather<T>(const cplx<T>*, cplx<T>*, const OlaGeom&, int64_t, cudaStream_t);
DGT_INST_OLA(float)
DGT_INST_OLA(double)

// =====================================================================================
// Real-signal coefficients: channels 0..M/2 of every column (Mh = M/2 + 1), and the full
// array back from them by conj(c(m, n)) = c((-m - 2 w(n)) mod M, n), 2 w(n) = (n lam1) mod lam2
// for lam2 <= 2.
// =====================================================================================
template <typename C>
__global__ void half_compact_kernel(const C* __restrict__ full, C* __restrict__ half, int64_t N, int64_t M,
                                    int64_t B) {
    const int64_t Mh = M / 2 + 1;
    const int64_t total = B * N * Mh;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e % Mh, r = e / Mh;
        half[e] = full[r * M + m];
    }
}

template <typename C>
__global__ void half_expand_kernel(const C* __restrict__ half, C* __restrict__ full, int64_t N, int64_t M,
                                   int64_t lam1, int64_t lam2, int64_t B) {
    const int64_t Mh = M / 2 + 1;
    const int64_t total = B * N * M;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t m = e % M, r = e / M;
        if (m < Mh) {
            full[e] = half[r * Mh + m];
        } else {
            const int64_t n = r % N;
            const int64_t two_w = ((n * lam1) % lam2) * (2 / lam2);
            int64_t pm = (-m - two_w) % M;
            if (pm < 0) pm += M;
            C v = half[r * Mh + pm];
            v.y = -v.y;
            full[e] = v;
        }
    }
}

template <typename T>
cudaError_t launch_half_compact(const cplx<T>* full, cplx<T>* half, int64_t N, int64_t M, int64_t B, cudaStream_t st) {
    const int64_t total = B * N * (M / 2 + 1);
    half_compact_kernel<cplx<T>><<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, st>>>(full, half, N, M, B);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_half_expand(const cplx<T>* half, cplx<T>* full, int64_t N, int64_t M, int64_t lam1, int64_t lam2,
                               int64_t B, cudaStream_t st) {
    const int64_t total = B * N * M;
    half_expand_kernel<cplx<T>><<<(unsigned)std::min<int64_t>((total + 255) / 256, 152 * 32), 256, 0, st>>>(
        half, full, N, M, lam1, lam2, B);
    return cudaGetLastError();
}
template cudaError_t launch_half_compact<float>(const float2*, float2*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_half_compact<double>(const double2*, double2*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_half_expand<float>(const float2*, float2*, int64_t, int64_t, int64_t, int64_t, int64_t,
                                               cudaStream_t);
template cudaError_t launch_half_expand<double>(const double2*, double2*, int64_t, int64_t, int64_t, int64_t, int64_t,
                                                cudaStream_t);

// =====================================================================================
// Batched transpose [B][R][Cc] -> [B][Cc][R] of complex arrays through 32 x 33 shared tiles
// (the two-dimensional transform applies each axis' plan to contiguous rows)
// =====================================================================================
template <typename C>
__global__ void __launch_bounds__(256) transpose_kernel(const C* __restrict__ in, C* __restrict__ out, int64_t R,
                                                        int64_t Cc) {
    __shared__ C tile[32][33];
    const int64_t b = blockIdx.z;
    const int64_t c0 = (int64_t)blockIdx.x * 32, r0 = (int64_t)blockIdx.y * 32;
    const C* src = in + b * R * Cc;
    C* dst = out + b * R * Cc;
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t r = r0 + i, cc = c0 + threadIdx.x;
        if (r < R && cc < Cc) tile[i][threadIdx.x] = src[r * Cc + cc];
    }
    __syncthreads();
    for (int i = threadIdx.y; i < 32; i += 8) {
        const int64_t cc = c0 + i, r = r0 + threadIdx.x;
        if (r < R && cc < Cc) dst[cc * R + r] = tile[threadIdx.x][i];
    }
}

template <typename T>
cudaError_t launch_transpose(const cplx<T>* in, cplx<T>* out, int64_t R, int64_t Cc, int64_t B, cudaStream_t st) {
    if (B <= 0 || R <= 0 || Cc <= 0) return cudaSuccess;
    dim3 grid((unsigned)((Cc + 31) / 32), (unsigned)((R + 31) / 32), (unsigned)B);
    transpose_kernel<cplx<T>><<<grid, dim3(32, 8), 0, st>>>(in, out, R, Cc);
    return cudaGetLastError();
}
template cudaError_t launch_transpose<float>(const float2*, float2*, int64_t, int64_t, int64_t, cudaStream_t);
template cudaError_t launch_transpose<double>(const double2*, double2*, int64_t, int64_t, int64_t, cudaStream_t);

// =====================================================================================
// Scratch of the allocation-free FIR synthesis entry point: one fixed array per GPU that
// loads the library, held until the process exits.  Host code must not use the symbol as
// a pointer: its device address comes from cudaGetSymbolAddress, looked up once per device.
// =====================================================================================
static __device__ __align__(256) unsigned char g_fir_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mu;
static std::map<int, void*> g_noalloc_addr;

cudaError_t noalloc_scratch(void** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    auto it = g_noalloc_addr.find(dev);
    if (it == g_noalloc_addr.end()) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fir_noalloc_scratch);
        if (e != cudaSuccess) return e;
        it = g_noalloc_addr.emplace(dev, p).first;
    }
    *out = it->second;
    return cudaSuccess;
}

// =====================================================================================
// Arithmetic throughput probe: every thread runs 8 independent fused multiply-add chains
// (scalar float, packed float pairs or double) for `iters` steps; the result is stored only
// when it equals a value no chain reaches, so the chains are not removed.
// =====================================================================================
template <int KIND>
__global__ void __launch_bounds__(256) fma_rate_kernel(int iters, float seed, float* out) {
    constexpr int K = 8;
    if constexpr (KIND == 0) {
        float a[K];
#pragma unroll
        for (int i = 0; i < K; ++i) a[i] = seed + (float)(threadIdx.x + i);
        const float x = 0.999f, y = 1e-3f;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < K; ++i) a[i] = fmaf(a[i], x, y);
        float sacc = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) sacc += a[i];
        if (sacc == -1.f) out[0] = sacc;
    } else if constexpr (KIND == 1) {
        float2 a[K];
#pragma unroll
        for (int i = 0; i < K; ++i) a[i] = make_float2(seed + (float)(threadIdx.x + i), seed - (float)i);
        const float2 x = make_float2(0.999f, 0.998f), y = make_float2(1e-3f, 2e-3f);
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < K; ++i) a[i] = __ffma2_rn(a[i], x, y);
        float sacc = 0.f;
#pragma unroll
        for (int i = 0; i < K; ++i) sacc += a[i].x + a[i].y;
        if (sacc == -1.f) out[0] = sacc;
    } else {
        double a[K];
#pragma unroll
        for (int i = 0; i < K; ++i) a[i] = (double)seed + (double)(threadIdx.x + i);
        const double x = 0.999, y = 1e-3;
        for (int it = 0; it < iters; ++it)
#pragma unroll
            for (int i = 0; i < K; ++i) a[i] = fma(a[i], x, y);
        double sacc = 0.0;
#pragma unroll
        for (int i = 0; i < K; ++i) sacc += a[i];
        if (sacc == -1.0) out[0] = (float)sacc;
    }
}

cudaError_t fma_rate(int kind, int iters, int blocks, float* out, cudaStream_t st, double* flops) {
    constexpr int K = 8, THR = 256;
    cudaEvent_t e0, e1;
    cudaError_t e = cudaEventCreate(&e0);
    if (e != cudaSuccess) return e;
    e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cudaEventDestroy(e0);
        return e;
    }
    auto launch = [&](int n) {
        if (kind == 0) fma_rate_kernel<0><<<blocks, THR, 0, st>>>(n, 1.f, out);
        else if (kind == 1) fma_rate_kernel<1><<<blocks, THR, 0, st>>>(n, 1.f, out);
        else fma_rate_kernel<2><<<blocks, THR, 0, st>>>(n, 1.f, out);
    };
    launch(iters / 8);                                      // warm-up
    cudaEventRecord(e0, st);
    launch(iters);
    cudaEventRecord(e1, st);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (e != cudaSuccess) return e;
    const double fmas = (double)blocks * THR * K * (double)iters * (kind == 1 ? 2.0 : 1.0);
    *flops = 2.0 * fmas / (ms * 1e-3);
    return cudaSuccess;
}

#define DGT_INST_AUX(T)                                                                                               \
    template cudaError_t launch_fir_analysis<T>(const void*, int, cplx<T>*, const FirParams<cplx<T>>&, const FftRef&, \
                                                int64_t, cudaStream_t);                                               \
    template cudaError_t launch_fir_synthesis<T>(const cplx<T>*, void*, int, cplx<T>*, const FirParams<cplx<T>>&,     \
                                                 const FftRef&, int64_t, cudaStream_t);                               \
    template cudaError_t launch_coset_windows<T>(const cplx<T>*, cplx<T>*, int64_t, int64_t, int64_t,                 \
                                                 const int64_t*, const CisTable<cplx<T>>&, cudaStream_t);             \
    template cudaError_t launch_chirp_table<T>(const ChirpParams<cplx<T>>&, cplx<T>*, cudaStream_t);                  \
    template cudaError_t launch_grad_window_combine<T>(const cplx<T>*, void*, int, int64_t, int64_t, int64_t,         \
                                                       const int64_t*, const CisTable<cplx<T>>&, cudaStream_t);       \
    template cudaError_t launch_logmag<T>(const cplx<T>*, cplx<T>*, double*, double*, int64_t, T, int64_t, cudaStream_t);

DGT_INST_AUX(float)
DGT_INST_AUX(double)
template cudaError_t launch_convert<double, float>(const void*, int, cplx<float>*, int64_t, cudaStream_t);
template cudaError_t launch_convert<double, double>(const void*, int, cplx<double>*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, double>(const void*, int, cplx<double>*, int64_t, cudaStream_t);
template cudaError_t launch_convert<float, float>(const void*, int, cplx<float>*, int64_t, cudaStream_t);

}  // namespace dgt
