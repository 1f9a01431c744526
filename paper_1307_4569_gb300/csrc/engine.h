// Internal interface between the host planner (plan.cpp) and the CUDA kernels.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "cplx.cuh"
#include "fft.cuh"

namespace dgt {

// Threads per CTA of the FFT-tile kernels, and the shared memory one CTA may use.
constexpr int kThreads = 256;
constexpr int kThreadsBig = 512;
constexpr size_t kSmemBudget = 200 * 1024;
inline int threads_for(int64_t elems) { return elems >= 4096 ? kThreadsBig : kThreads; }

struct FftRef {                 // one FFT length: radix plan + device twiddle table
    FftPlanDev pl;
    const void* tw;             // cplx<T>[n], tw[e] = exp(-2 pi i e / n)
};

// Separable lattice on which the Zak/polyphase engine runs (eqs. cd, pq).
struct SepGeom {
    int64_t L, a, M, b, N, c, d, p, q, K0;   // K0 = L / d = c p q
};

// Post-processing of the channel FFT (analysis) / pre-processing of its adjoint.
enum PostMode : int {
    POST_PLAIN = 0,     // separable lattice: row n -> column n
    POST_COSET = 1,     // row (j, nt) -> column lam2 nt + j, phase exp(-2 pi i nt at sigma_j / L)
    POST_SHEAR0 = 2,    // time shear only (s0 = 0): phase E_n, cyclic rotation of the column
    POST_SHEAR1 = 3,    // frequency shear (s0 != 0): phase E(k, m) and reindex of both indices
};

template <typename C> struct PostParams {
    int mode;
    int64_t L, M, N, b, a;            // output (nonseparable) lattice
    int64_t lam2, at;                 // coset
    const int64_t* sigma;             // coset frequency shifts sigma_j (device, J entries)
    int64_t s1a_modL;                 // shear0: (s1 * a) mod L ; rotation rot_n = floor(((-s1 a n) mod L)/b)
    int64_t C1_2N;                    // shear0: C1 mod 2N
    // shear1 (Algorithm 1, s0 != 0), all reduced modulo 2N or L as used
    int64_t Nr, C1, C2_N, C1_2N_, C2_2N, C3_2N, C4_2N, C5_2N, s1ar_L, C6_L;
    CisTable<C> cisL;                 // exp(2 pi i e / L)
    CisTable<C> cis2N;                // exp(2 pi i e / (2N)) = exp(pi i e / N)
    ModU64 mL, mN, m2N;               // reductions modulo L, N, 2N
    ModU64 mb;                        // division by b
    ModU64 mJN, mNs;                  // row = (b J + j) Ns + n of Y: division by J Ns and Ns (set by the launchers)
    int64_t lam1;                     // w(n) of the output columns (real-signal coefficients)
    int half;                         // coefficients hold channels 0..M/2 only (real signals, lam2 <= 2)
    // shear1 in 32-bit arithmetic (host-checked: (2N)^2 and L Nr below 2^32): the constants
    // above reduced to 32 bits and the reductions modulo 2N, L and the division by b
    int sh1_fast;
    uint32_t f_Nr, f_N, f_M, f_C1, f_C2, f_C3, f_C4, f_C5, f_s1ar, f_C6;
    ModU32 q2N, qL, qb;
};

// Signal pre-processing inside the factorisation / FFT_L passes.
enum PreMode : int {
    PRE_NONE = 0,
    PRE_CHIRP = 1,      // x(l) * exp(pi i (s l^2 (L+1) mod 2L) / L)   (pchirp(L, s))
};

template <typename C> struct ChirpParams {
    int mode;
    int64_t L;
    int64_t s_2L;                     // s mod 2L
    int conj;                         // multiply by the conjugate chirp
    CisTable<C> cis2L;                // exp(2 pi i e / (2L))
    ModU64 m2L;                       // reduction modulo 2L
    const C* tab;                     // the unconjugated chirp at l < L when the plan built it, else null
};

// ------------------------------------------------------------------------------------
// launchers (templated on the real type T; explicitly instantiated in the .cu files)
// ------------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_zak_fwd(const void* src, int src_real, int64_t src_bstride, cplx<T>* zf, int64_t zf_bstride,
                           int64_t L, int64_t d, const FftRef& fd, const ChirpParams<cplx<T>>& pre, int64_t B,
                           cudaStream_t st);

template <typename T>
cudaError_t launch_prod_ifft(const cplx<T>* zf, const cplx<T>* zg, int64_t J, cplx<T>* y, const SepGeom& g,
                             const FftRef& fd, int64_t B, cudaStream_t st);

template <typename T>
cudaError_t launch_fft_post(const cplx<T>* y, cplx<T>* c, const SepGeom& g, int64_t J, const FftRef& fm,
                            const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st);

// adjoint chain (synthesis)
template <typename T>
cudaError_t launch_pre_ifft(const cplx<T>* c, cplx<T>* y, const SepGeom& g, int64_t J, const FftRef& fm,
                            const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st);

template <typename T>
cudaError_t launch_fft_prod_adj(const cplx<T>* y, const cplx<T>* zg, int64_t J, cplx<T>* zf, const SepGeom& g,
                                const FftRef& fd, int64_t B, unsigned int* expired, cudaStream_t st);

template <typename T>
cudaError_t launch_zak_inv(const cplx<T>* zf, int64_t zf_bstride, void* dst, int dst_real, int64_t dst_bstride,
                           int64_t L, int64_t d, const FftRef& fd, const ChirpParams<cplx<T>>& post, T scale,
                           int64_t B, cudaStream_t st);

// window gradient through the factorisation: V_j[xi][col] accumulated over the batch
// (part: scratch of fft_grad_window_groups() J L elements for the per-group sums, or null for one group)
template <typename T>
cudaError_t launch_fft_grad_window(const cplx<T>* y, const cplx<T>* zf, int64_t J, cplx<T>* v, cplx<T>* part,
                                   const SepGeom& g, const FftRef& fd, int64_t B, cudaStream_t st);
int64_t fft_grad_window_groups(const SepGeom& g, int64_t J, int64_t B, size_t elem);

// four-step FFT of length L = L1 * L2 (frequency-shear branch and window set-up)
template <typename T>
cudaError_t launch_fftL_cols(const void* src, int src_real, cplx<T>* tmp, int64_t L1, int64_t L2, int dir,
                             const FftRef& f1, const ChirpParams<cplx<T>>& pre, const CisTable<cplx<T>>& cisL,
                             int64_t B, cudaStream_t st);
template <typename T>
cudaError_t launch_fftL_rows(const cplx<T>* tmp, void* dst, int dst_real, int64_t L1, int64_t L2, int dir,
                             const FftRef& f2, const ChirpParams<cplx<T>>& post, T scale, int64_t B,
                             cudaStream_t st);

// FIR (weighted overlap-add) path
template <typename C> struct FirParams {
    int64_t L, a, M, N, lam1, lam2, Lg, center;
    const C* taps;                    // Lg taps of the analysis / synthesis window
    CisTable<C> cisLM;                // exp(2 pi i e / (lam2 M))
    // [lam2][Lg] modulated taps conj(h(t)) exp(-2 pi i t wn / (lam2 M)), wn = (n lam1) mod lam2.
    // With l = ln + t (ln = time of tap 0 of column n) the modulation exp(-2 pi i l w(n)/M) of
    // the definition splits into this tap factor and the column constant
    // exp(-2 pi i ln wn / (lam2 M)), applied once per column after (before) the FFT.
    const C* mtaps;
    const typename RealOf<C>::type* rtaps;   // Re mtaps[0][.], dense (Lg values)
    ModU64 mN;                        // division by N (row = b N + n)
    int64_t cols;                     // time positions per CTA
    int64_t group;                    // rows transformed at once (spare buffer rows)
    int half;                         // coefficients hold channels 0..M/2 only (real signals, lam2 <= 2)
    int pairable;                     // the window of these taps is real: real-input pairing applies
    const C* hb;                      // exp(-pi i k / M), k < M (lam2 = 2; real-input pairing)
};
template <typename T>
cudaError_t launch_fir_analysis(const void* f, int f_real, cplx<T>* c, const FirParams<cplx<T>>& fp,
                                const FftRef& fm, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t launch_fir_synthesis(const cplx<T>* c, void* f, int f_real, cplx<T>* seams,
                                 const FirParams<cplx<T>>& fp, const FftRef& fm, int64_t B, cudaStream_t st);
template <typename C>
int64_t fir_seam_elems(const FirParams<C>& fp);
// modulated taps (see FirParams::mtaps) from float64 taps h[Lg]; exact integer phase reduction
template <typename T>
cudaError_t launch_fir_modtaps(const double2* h, cplx<T>* out, int64_t Lg, int64_t lam2, int64_t M, cudaStream_t st);

// blockwise (overlap-add) DGT: block length Lb, Nb blocks, local length Lx with Nx columns;
// S = Lb / a global columns per block; local columns 0..nu_hi keep their offset, the rest stand
// for offset nu - Nx; K = blocks that can reach one global column (at most Nb)
struct OlaGeom {
    int64_t L, a, M, N, Lb, Nb, Lx, Nx, S, nu_hi, K;
};
template <typename T>
cudaError_t launch_ola_split(const void* f, int f_real, void* x, const OlaGeom& og, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t launch_ola_take(const void* y, int f_real, void* f, const OlaGeom& og, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t launch_ola_add(const cplx<T>* cx, cplx<T>* c, const OlaGeom& og, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t launch_ola_gather(const cplx<T>* c, cplx<T>* cx, const OlaGeom& og, int64_t B, cudaStream_t st);

// real-signal coefficients: channels 0..M/2 (compact) and the full array back (expand)
template <typename T>
cudaError_t launch_half_compact(const cplx<T>* full, cplx<T>* half, int64_t N, int64_t M, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t launch_half_expand(const cplx<T>* half, cplx<T>* full, int64_t N, int64_t M, int64_t lam1, int64_t lam2,
                               int64_t B, cudaStream_t st);

// batched transpose [B][R][Cc] -> [B][Cc][R]
template <typename T>
cudaError_t launch_transpose(const cplx<T>* in, cplx<T>* out, int64_t R, int64_t Cc, int64_t B, cudaStream_t st);

// elementwise helpers
template <typename T>
cudaError_t launch_coset_windows(const cplx<T>* g, cplx<T>* gj, int64_t L, int64_t a, int64_t J, const int64_t* sigma,
                                 const CisTable<cplx<T>>& cisL, cudaStream_t st);
template <typename T>
cudaError_t launch_chirp_table(const ChirpParams<cplx<T>>& cp, cplx<T>* tab, cudaStream_t st);
template <typename Tin, typename Tout>
cudaError_t launch_convert(const void* in, int in_real, cplx<Tout>* out, int64_t n, cudaStream_t st);
template <typename T>
cudaError_t launch_grad_window_combine(const cplx<T>* wj, void* grad, int grad_real, int64_t L, int64_t a, int64_t J,
                                       const int64_t* sigma, const CisTable<cplx<T>>& cisL, cudaStream_t st);
template <typename T>
cudaError_t launch_logmag(const cplx<T>* c, cplx<T>* u, double* partial, double* loss, int64_t n, T eps, int64_t B,
                          cudaStream_t st);

// dual / tight window Gram blocks (float64)
cudaError_t launch_gram_solve(const double2* zg, int64_t J, double2* zout, const SepGeom& g, int tight,
                              int* status, cudaStream_t st);
cudaError_t launch_fir_dual(const double2* taps, double2* out, int64_t Lg, int64_t a, int64_t M, int tight,
                            int* status, cudaStream_t st);

// Fixed scratch for the allocation-free FIR synthesis entry point (bytes per GPU), and its
// device address on the current device (looked up on the first call per device).
constexpr size_t kNoAllocScratchBytes = (size_t)4 << 20;
cudaError_t noalloc_scratch(void** out);

// FFT self-test (batched transforms along contiguous rows)
template <typename T>
cudaError_t launch_fft_rows_test(const cplx<T>* in, cplx<T>* out, const FftRef& f, int dir, int64_t rows,
                                 cudaStream_t st);

// Power-of-two fast path (kernels_p2.cuh); each returns cudaErrorNotSupported when the length
// or geometry is outside it, and the caller then uses the generic kernel.
template <typename T>
cudaError_t p2_zak_fwd(const void* src, int src_real, int64_t sbs, cplx<T>* zf, int64_t zbs, int64_t d, int64_t K0,
                       const void* tw, const ChirpParams<cplx<T>>& pre, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t p2_prod_ifft(const cplx<T>* zf, const cplx<T>* zg, int64_t J, cplx<T>* y, const SepGeom& g, const void* tw,
                         int64_t B, cudaStream_t st);
template <typename T>
cudaError_t p2_fft_prod_adj(const cplx<T>* y, const cplx<T>* zg, int64_t J, cplx<T>* zf, const SepGeom& g,
                            const void* tw, int64_t B, unsigned int* expired, cudaStream_t st);
template <typename T>
cudaError_t p2_zak_inv(const cplx<T>* zf, int64_t zbs, void* dst, int dst_real, int64_t dbs, int64_t d, int64_t K0,
                       const void* tw, const ChirpParams<cplx<T>>& post, T scale, int64_t B, cudaStream_t st);
// mixed-radix row kernels (kernels_mr.cuh): cudaErrorNotSupported for a length without a
// compiled transform
template <typename T>
cudaError_t mr_fft_post(const cplx<T>* y, cplx<T>* c, const SepGeom& g, int64_t J, const void* tw,
                        const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t mr_pre_ifft(const cplx<T>* c, cplx<T>* y, const SepGeom& g, int64_t J, const void* tw,
                        const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t mr_zak_fwd(const void* src, int src_real, int64_t sbs, cplx<T>* zf, int64_t zbs, int64_t d, int64_t K0,
                       const void* tw, const ChirpParams<cplx<T>>& pre, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t mr_prod_ifft(const cplx<T>* zf, const cplx<T>* zg, int64_t J, cplx<T>* y, const SepGeom& g,
                         const void* tw, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t mr_fft_prod_adj(const cplx<T>* y, const cplx<T>* zg, int64_t J, cplx<T>* zf, const SepGeom& g,
                            const void* tw, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t mr_zak_inv(const cplx<T>* zf, int64_t zbs, void* dst, int dst_real, int64_t dbs, int64_t d, int64_t K0,
                       const void* tw, const ChirpParams<cplx<T>>& post, T scale, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t mr_fftL_cols(const void* src, int src_real, cplx<T>* tmp, int64_t L1, int64_t L2, int dir, const void* tw,
                         const ChirpParams<cplx<T>>& pre, const CisTable<cplx<T>>& cisL, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t mr_fftL_rows(const cplx<T>* tmp, void* dst, int dst_real, int64_t L1, int64_t L2, int dir, const void* tw,
                         const ChirpParams<cplx<T>>& post, T scale, int64_t B, cudaStream_t st);
// the lengths with a compiled mixed-radix transform (the cases of MR_SWITCH in kernels_mr.cuh)
inline bool mr_compiled_len(int64_t n) {
    switch (n) {
        case 60: case 120: case 180: case 240: case 360: case 480: case 720: case 960: case 2160: return true;
        default: return false;
    }
}
// Bounded device waits (the tensor-copy staging of fft_prod_adj): the wait limit in clock
// cycles that launches pass to the kernels (a test hook lowers it).  A CTA whose wait expires
// sets the caller's word `expired` to 1 (a plan's host-mapped word, or the word at the start
// of a caller workspace), so each expiry is traced to the plan or workspace of its launch.
// arithmetic throughput probe: kind 0 scalar float FMA, 1 packed float pairs, 2 double FMA;
// `blocks` CTAs of 256 threads, 8 chains of `iters` FMAs per thread; flop/s (2 per FMA lane)
cudaError_t fma_rate(int kind, int iters, int blocks, float* out, cudaStream_t st, double* flops);
constexpr long long kWaitCycles = 2000000000LL;       // about a second
extern long long g_wait_limit_cycles;
// columns per chunk of the power-of-two FIR synthesis for FFT length M (0: not applicable)
template <typename T> int64_t p2_fir_synthesis_cols(int64_t M, int64_t N, int64_t a, int64_t Lg);
// lengths of the power-of-two column kernels
inline bool p2_col_len_ok(int64_t n) { return n >= 128 && n <= 8192 && (n & (n - 1)) == 0; }
// fused Zak analysis (p = 1): zak_fwd + prod_ifft
template <typename T>
cudaError_t p2_zak_prod_ifft(const void* src, int src_real, int64_t sbs, const cplx<T>* zg, int64_t J, cplx<T>* y,
                             const SepGeom& g, const void* tw, const ChirpParams<cplx<T>>& pre, int64_t B,
                             cudaStream_t st);
template <typename T>
cudaError_t p2_fft_post(const cplx<T>* y, cplx<T>* c, const SepGeom& g, int64_t J, const void* tw,
                        const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t p2_pre_ifft(const cplx<T>* c, cplx<T>* y, const SepGeom& g, int64_t J, const void* tw,
                        const PostParams<cplx<T>>& pp, int64_t B, cudaStream_t st);
template <typename T>
cudaError_t p2_fir_analysis(const void* f, int f_real, cplx<T>* c, const FirParams<cplx<T>>& fp, const void* tw,
                            int64_t B, cudaStream_t st);
template <typename T>
cudaError_t p2_fir_synthesis(const cplx<T>* c, void* f, int f_real, cplx<T>* seams, const FirParams<cplx<T>>& fp,
                             const void* tw, int64_t B, cudaStream_t st);

// CTA sizing: largest FFT tile (elements, two ping-pong buffers) that fits the budget
template <typename T> constexpr int64_t tile_cap() { return (int64_t)(kSmemBudget / (2 * sizeof(cplx<T>))); }

}  // namespace dgt
