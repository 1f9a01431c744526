/*
 * dgt.h -- discrete Gabor transform on a nonseparable lattice, CUDA (sm_103a) library.
 *
 * The transform (Wiesmeyr, Holighaus, Soendergaard, "Efficient algorithms for discrete
 * Gabor transforms on a nonseparable lattice", Section 2.1, eq. DGT):
 *
 *   c(m, n) = sum_{l<L} f(l) conj(g(l - a n)) exp(-2 pi i l (m + w(n)) / M),
 *   w(n)    = ((n * lambda1) mod lambda2) / lambda2,      m < M,  n < N = L / a,
 *
 * i.e. the samples of the short-time Fourier transform on the lattice
 * {(a n, m b + s(n))}, b = L / M, s(n) = (n s) mod b, s = b lambda1 / lambda2
 * (Prop. lattNF).  Synthesis is the adjoint (Section 2.1, inversion formula):
 *
 *   f(l) = sum_{m,n} c(m, n) gamma(l - a n) exp(+2 pi i l (m + w(n)) / M).
 *
 * Conventions for every entry point
 *   - Buffers passed to dgt_exec / idgt_exec / the window routines are DEVICE pointers
 *     on the current CUDA device, owned by the caller, and must not overlap.
 *   - Signals are [batch][L]; real signals are float32/float64, complex signals are
 *     interleaved (re, im) pairs of the plan's precision.  Coefficients are
 *     [batch][N][M] complex, m contiguous (column c(., n) is contiguous).
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is enqueued
 *     asynchronously; no entry point synchronises the stream unless stated.
 *   - Return value: DGT_OK or a dgt_status code; dgt_last_error() gives a message.
 *     Asynchronous device faults surface at the next call that synchronises.  An expired
 *     bounded device wait of a plan's earlier synthesis (see dgt_plan_status) is returned as
 *     DGT_ERR_TIMEOUT by that plan's next call, which then enqueues nothing.
 *   - A plan is not thread-safe: use one plan per host thread or serialise calls.
 */
#ifndef DGT_H
#define DGT_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dgt_plan_s* dgt_plan_t;

typedef enum {
    DGT_OK = 0,
    DGT_ERR_ARG = 1,          /* invalid argument (null pointer, bad enum, lambda1 >= lambda2, ...) */
    DGT_ERR_LENGTH = 2,       /* L is not a multiple of lambda2 * lcm(a, M) (Prop. minsig) */
    DGT_ERR_NOT_FRAME = 3,    /* a Gram block is singular or ill-conditioned: no dual / tight window */
    DGT_ERR_CUDA = 4,         /* a CUDA call failed */
    DGT_ERR_OOM = 5,          /* device allocation failed */
    DGT_ERR_TIMEOUT = 6,      /* a bounded device wait expired */
    DGT_ERR_UNSUPPORTED = 7   /* valid lattice outside this build's limits (FFT length, Gram block size) */
} dgt_status;

typedef enum {
    DGT_ROUTE_AUTO = 0,       /* FIR windows: FIR route; full windows: shear if s0 = 0, else coset */
    DGT_ROUTE_COSET = 1,      /* union of lambda2 separable lattices (Prop. mwindec, eq. mw_phases) */
    DGT_ROUTE_SHEAR = 2,      /* chirps + separable DGT + phase / reindex (Theorem shearform, Algorithm 1) */
    DGT_ROUTE_FIR = 3         /* weighted overlap-add with a short window (eq. rect-flops-FIR) */
} dgt_route;

typedef enum { DGT_F32 = 0, DGT_F64 = 1 } dgt_precision;

typedef enum {
    DGT_WINDOW_FULL = 0,      /* len == L samples, g(0) first */
    DGT_WINDOW_FIR = 1        /* len <= L/2 taps; tap t sits at time (t - center) mod L */
} dgt_window_kind;

typedef enum {
    DGT_SYN_ADJOINT = 0,      /* window g itself: the adjoint C_g^* */
    DGT_SYN_DUAL = 1,         /* canonical dual S^{-1} g: perfect reconstruction */
    DGT_SYN_TIGHT = 2         /* canonical tight S^{-1/2} g, with the analysis done by the same tight window */
} dgt_synthesis_window;

typedef struct {
    int kind;                 /* dgt_window_kind */
    int64_t len;              /* number of samples / taps */
    int64_t center;           /* FIR only: index of the tap at time 0 */
    const double* data;       /* HOST memory, float64: len reals, or len interleaved complex pairs */
    int is_real;              /* 1: data holds len reals */
} dgt_window;

typedef struct {
    int64_t L, a, M, lambda1, lambda2, b, N, s;
    int route;                /* resolved route (never DGT_ROUTE_AUTO) */
    int precision;
    int64_t s0, s1, b_r;      /* shear parameters chosen for the shear route (0 otherwise) */
    int64_t sep_a, sep_M;     /* separable lattice run by the Zak engine (coset: lambda2 a, M) */
    int64_t c, d, p, q;       /* its constants, eqs. (cd, pq) */
    int64_t n_windows;        /* window factors held (lambda2 for coset, 1 otherwise) */
    int64_t fir_len;          /* FIR taps (FIR route) */
    int64_t ola_block;        /* blockwise plans: block length Lb (0 otherwise) */
    int64_t ola_len;          /* blockwise plans: length Lx of the blocks' transforms */
} dgt_plan_info;

/* Create a plan for the lattice (L, a, M, lambda1/lambda2) and window g.
 * Checks feasibility (Prop. minsig: L multiple of lambda2 * lcm(a, M)), chooses the route,
 * finds the shear parameters (Theorem shearform, eq. modcond) and precomputes on the device
 * the window's factorisation.  Copies g; *plan receives the handle.  Synchronises `stream`.
 * Errors: DGT_ERR_ARG, DGT_ERR_LENGTH, DGT_ERR_UNSUPPORTED, DGT_ERR_OOM, DGT_ERR_CUDA. */
int dgt_plan_create(dgt_plan_t* plan, int64_t L, int64_t a, int64_t M, int64_t lambda1, int64_t lambda2,
                    const dgt_window* g, int route, int precision, void* stream);

/* Blockwise (overlap-add) plan for an FIR window: Section 4 (the OLA algorithm) and Section 4.1
 * (the shear-OLA algorithm).  The signal is cut into L / block_len blocks; each block,
 * zero-extended to Lx = the smallest multiple of lambda2 * lcm(a, M) not below
 * block_len + g->len whose transform this build supports (reported as ola_len by
 * dgt_plan_get_info), is transformed by a full-window plan of length Lx (inner_route:
 * DGT_ROUTE_COSET, DGT_ROUTE_SHEAR, or DGT_ROUTE_AUTO for shear when s0 = 0, else coset),
 * and the blocks' coefficient columns are added into the columns of the length-L
 * transform; synthesis is the adjoint (gather the columns, synthesise each block, keep its
 * block_len samples).  The results equal those of dgt_plan_create with the same FIR window;
 * the cost grows by rho = Lx / block_len (eq. OLA-eff).  The handle works with dgt_exec,
 * dgt_exec_ws, idgt_exec, idgt_exec_ws (adjoint, and dual / tight for windows no longer
 * than M), dgt_window_dual / _tight (length-L windows), dgt_workspace_bytes, dgt_plan_bytes,
 * dgt_plan_status, dgt_plan_get_info and dgt_plan_destroy; the other entry points return
 * DGT_ERR_UNSUPPORTED or DGT_ERR_ARG.  Synchronises `stream`.
 * Errors: DGT_ERR_ARG (not an FIR window, block shorter than the window, FIR inner route),
 * DGT_ERR_LENGTH (L or block_len not a multiple of lambda2 * lcm(a, M), block_len not
 * dividing L, Lx > L), and those of dgt_plan_create for the blocks' plan. */
int dgt_plan_create_ola(dgt_plan_t* plan, int64_t L, int64_t a, int64_t M, int64_t lambda1, int64_t lambda2,
                        const dgt_window* g, int64_t block_len, int inner_route, int precision, void* stream);

/* Two-dimensional DGT on a tensor-product lattice Lambda1 x Lambda2 with a separable window
 * g1 (x) g2 (Section 3.5, extension to higher dimensions): each axis is a lattice of its own
 * (L_i, a_i, M_i, lambda_i1 / lambda_i2, window g_i, one dgt_plan_create each, same route
 * and precision), and the transform is the second axis' DGT of every row followed by the
 * first axis' DGT of every column.  Signals f: DEVICE [batch][L1][L2] (real or complex);
 * coefficients c: DEVICE [batch][N1][M1][N2][M2] complex, i.e. c(m1, n1, m2, n2) at
 * ((n1 M1 + m1) N2 + n2) M2 + m2.  idgt2_exec: synthesis with g1 (x) g2 (adjoint), or the
 * tensor product of the axes' dual / tight windows (which_window as for idgt_exec).
 * Work arrays (2 B L1 N2 M2 + B N1 M1 N2 M2 complex) are plan-owned.  Errors: those of
 * dgt_plan_create for either axis, and of dgt_exec / idgt_exec. */
typedef struct dgt2_plan_s* dgt2_plan_t;
int dgt2_plan_create(dgt2_plan_t* plan, int64_t L1, int64_t a1, int64_t M1, int64_t lambda11, int64_t lambda12,
                     const dgt_window* g1, int64_t L2, int64_t a2, int64_t M2, int64_t lambda21, int64_t lambda22,
                     const dgt_window* g2, int route, int precision, void* stream);
int dgt2_exec(dgt2_plan_t plan, const void* f, int f_is_real, void* c, int64_t batch, void* stream);
int idgt2_exec(dgt2_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window, void* stream);
/* Synchronise `stream` and report a pending asynchronous error of either axis' work. */
int dgt2_plan_status(dgt2_plan_t plan, void* stream);
/* Release the plan (synchronises the device first). */
void dgt2_plan_destroy(dgt2_plan_t plan);

/* Copy the resolved plan parameters into *info. */
int dgt_plan_get_info(dgt_plan_t plan, dgt_plan_info* info);

/* Replace the window with a DEVICE buffer of the plan's precision (same kind and length as at
 * creation; real or interleaved complex) and recompute its factorisation.  Invalidates the
 * cached dual / tight windows.  Asynchronous on `stream`. */
int dgt_plan_set_window(dgt_plan_t plan, const void* g_dev, int is_real, void* stream);

/* Analysis: c = C_g f for `batch` signals (Section 2.1, eq. DGT; coset route eqs. mw_frop /
 * mw_phases, shear route Algorithm 1, FIR route eq. rect-flops-FIR).
 * f: [batch][L] real (f_is_real = 1) or complex; c: [batch][N][M] complex.
 * Uses the plan's workspace (grown on demand with cudaMalloc; see dgt_exec_ws). */
int dgt_exec(dgt_plan_t plan, const void* f, int f_is_real, void* c, int64_t batch, void* stream);

/* Synthesis: f = C_gamma^* c, gamma chosen by `which_window` (dgt_synthesis_window).
 * The dual / tight window is computed on first use (Gram blocks in float64) and cached.
 * f_real_out = 1 writes the real part only (float of the plan precision). */
int idgt_exec(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window,
              void* stream);

/* Synthesis with a window of the caller's choosing (Section 2.1, inversion formula with an
 * arbitrary synthesis window gamma: f(l) = sum_{m,n} c(m, n) gamma(l - a n)
 * exp(+2 pi i l (m + w(n)) / M)).  gamma: DEVICE buffer of the plan's precision, real
 * (gamma_is_real = 1) or interleaved complex; L samples for the coset and shear routes, or the
 * plan's Lg taps (same centre as the analysis window) for the FIR route.  The window's
 * factorisation is rebuilt on `stream` at every call (one transform of gamma, O(L log L);
 * plan-owned memory, grown with cudaMalloc on first use), so the call may allocate.
 * Errors: DGT_ERR_UNSUPPORTED for blockwise plans, and those of idgt_exec. */
int idgt_exec_window(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, const void* gamma,
                     int gamma_is_real, void* stream);

/* Real-signal coefficients (the real-signal variant of the interface, Section 4.4): for a real
 * signal and a real window on a lattice with lambda2 <= 2 and M even,
 * c(m, n) = conj(c((-m - 2 w(n)) mod M, n)), so the channels 0..M/2 determine c.
 * dgt_exec_real: f DEVICE [batch][L] real -> c DEVICE [batch][N][M/2 + 1] complex.
 * idgt_exec_real: the synthesis of the full coefficients those channels stand for, real
 * output [batch][L]; which_window as for idgt_exec.  Both stage the full array in
 * plan-owned memory (one call at a time per plan).
 * Errors: DGT_ERR_UNSUPPORTED (lambda2 > 2, odd M, complex window), and those of
 * dgt_exec / idgt_exec. */
int dgt_exec_real(dgt_plan_t plan, const void* f, void* c, int64_t batch, void* stream);
int idgt_exec_real(dgt_plan_t plan, const void* c, void* f, int64_t batch, int which_window, void* stream);

/* As dgt_exec / idgt_exec (the same transforms, eq. (DGT) and its adjoint), with HOST
 * buffers: f HOST [batch][L], c HOST [batch][N][M], in the layouts of dgt_exec / idgt_exec.
 * The batch goes in chunks of `chunk` signals (0: the whole batch) through two plan-owned
 * device staging slots.  The host-to-device copy of chunk i + 1 and the device-to-host copy of
 * chunk i - 1 run on two plan-owned streams while chunk i is transformed on `stream`.  The
 * call is ordered after earlier work on `stream`, and later work on `stream` waits for its last
 * copy; with pinned (page-locked) host buffers it returns before the copies end, so
 * synchronise `stream` before reading the output.  Pageable buffers work, with copies that
 * block the host.  The staging slots grow to 2 chunks of input and output and stay with the
 * plan.  One call at a time per plan, with the plan's device current.  Errors: DGT_ERR_ARG
 * (null pointer, negative batch or chunk, another device current), and those of dgt_exec /
 * idgt_exec. */
int dgt_exec_host(dgt_plan_t plan, const void* f, int f_is_real, void* c, int64_t batch, int64_t chunk,
                  void* stream);
int idgt_exec_host(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window,
                   int64_t chunk, void* stream);

/* Workspace needed by dgt_exec_ws / idgt_exec_ws for `batch` signals, in bytes. */
int dgt_workspace_bytes(dgt_plan_t plan, int64_t batch, size_t* bytes);

/* As dgt_exec / idgt_exec, with a caller-provided device workspace of at least
 * dgt_workspace_bytes(batch) bytes, 256-byte aligned.  These never allocate (the dual /
 * tight window of idgt_exec_ws must already be cached by dgt_window_dual / _tight).
 * The first word of the workspace is the call's expiry word: idgt_exec_ws clears it in
 * stream order before its kernels, and a kernel whose bounded wait expires sets it;
 * dgt_workspace_status reads it.  Calls on different streams with different workspaces
 * may run concurrently; calls sharing a workspace must be ordered. */
int dgt_exec_ws(dgt_plan_t plan, const void* f, int f_is_real, void* c, int64_t batch, void* workspace,
                void* stream);
int idgt_exec_ws(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window,
                 void* workspace, void* stream);

/* Canonical dual window S^{-1} g (eq. frameop) into gamma_out: L complex values of the plan's
 * precision (device).  Computed through the Zak-domain Gram blocks of the coset decomposition
 * (eq. mw_frop), inverted in float64; FIR windows no longer than M use the diagonal form.
 * DGT_ERR_NOT_FRAME if a block is singular.  Synchronises `stream`. */
int dgt_window_dual(dgt_plan_t plan, void* gamma_out, void* stream);

/* Canonical tight window S^{-1/2} g, as dgt_window_dual. */
int dgt_window_tight(dgt_plan_t plan, void* gt_out, void* stream);

/* Window gradient of a real-valued loss l(c): given G = dl/dRe(c) + i dl/dIm(c) for every
 * coefficient of `batch` signals f, writes grad_g = sum over the batch of
 * sum_n f(. + a n) conj(U_n(. + a n)), U_n(l) = sum_m G(m,n) exp(+2 pi i l (m + w(n))/M)
 * (L values, real part if grad_real).  The signal gradient is idgt_exec(..., DGT_SYN_ADJOINT)
 * applied to G.  Full-length windows only. */
int dgt_grad_window(dgt_plan_t plan, const void* f, int f_is_real, const void* G, void* grad_g, int grad_real,
                    int64_t batch, void* stream);

/* Allocation-free FIR synthesis.  For callers that must not allocate device memory while
 * they run -- a real-time audio callback cannot wait on cudaMalloc, which may synchronise the
 * device and take driver locks; a plug-in host may own all device memory; a process may have
 * fenced off its allocation budget.  Same result as idgt_exec on an FIR-route plan, but the
 * scratch that holds the overlap seams between neighbouring column chunks lives in one fixed
 * 4 MiB array that the library keeps on every GPU that loads it, until the process exits; the
 * seams need batch * (N / chunk columns) * 2 * (Lg - a) complex values, and a call needing
 * more than 4 MiB returns DGT_ERR_UNSUPPORTED.  Nothing in the array has to start at zero:
 * each call writes every scratch element it later reads.  All calls share the array, so calls
 * that overlap on the GPU (other streams, other threads) race; serialise them.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress): make that first
 * call before any stream capture.  The dual / tight window must already be cached
 * (dgt_window_dual / dgt_window_tight), else DGT_ERR_ARG.  The paper has no counterpart:
 * this is a deployment variant of the weighted overlap-add synthesis. */
int dgt_fir_synthesis_noalloc(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch,
                              int which_window, void* stream);

/* Log-magnitude loss helper: loss_b = sum log(|c|^2 + eps) per signal (float64, device array of
 * `batch`), and G = 2 c / (|c|^2 + eps) (device, may be NULL). */
int dgt_logmag_loss(dgt_plan_t plan, const void* c, void* G, double* loss_dev, double eps, int64_t batch,
                    void* stream);

/* Bytes of device memory owned by the plan (tables, window factors, cached windows, workspace). */
int dgt_plan_bytes(dgt_plan_t plan, size_t* bytes);

/* Synchronise `stream` and report a pending asynchronous CUDA error of this plan's work
 * as DGT_ERR_CUDA, or DGT_ERR_TIMEOUT when a bounded device wait of this plan's calls
 * without a caller workspace expired since the last check (each plan has its own expiry
 * word; dgt_workspace_status covers the calls with a caller workspace).  (No kernel of this library waits on another one.  The one device wait is the
 * float synthesis kernel's wait for the tile copies it issued itself: a CTA whose wait
 * exceeds the limit of dgt_wait_limit lets its copies land, records the expiry and returns,
 * leaving its part of the output unwritten; the context stays usable.) */
int dgt_plan_status(dgt_plan_t plan, void* stream);

/* Synchronise `stream` and report a pending asynchronous CUDA error as DGT_ERR_CUDA, or an
 * expired bounded wait of any live plan's calls without a caller workspace as
 * DGT_ERR_TIMEOUT (clearing those plans' words). */
int dgt_sync(void* stream);

/* Synchronise `stream` (the one the idgt_exec_ws call ran on) and report DGT_ERR_TIMEOUT when
 * a kernel of the last synthesis that used `workspace` gave up waiting for its tile copies
 * (its output is then incomplete), clearing the word; DGT_ERR_CUDA for a pending CUDA
 * error.  A serving loop calls it per batch to attribute an expiry to that batch. */
int dgt_workspace_status(dgt_plan_t plan, const void* workspace, void* stream);

/* Test hook: the limit, in SM clock cycles, of the bounded device waits of later launches
 * (default 2e9, about a second).  cycles = 0 makes every wait expire at once, so that the
 * error path can be tested without a fault; cycles < 0 only queries.  Returns the previous
 * limit.  Host-global: it applies to every plan of the process. */
long long dgt_wait_limit(long long cycles);

/* The largest total size in bytes of the chirp tables that a shear-route plan created later
 * keeps (Algorithm 1's pchirp factors, one table of L complex values per chirp, computed from
 * the exact integer exponent; default 2^30).  A plan whose tables would exceed it computes the
 * factors per sample instead, with bit-identical results.  bytes < 0 only queries.  Returns the
 * previous cap.  Host-global. */
long long dgt_chirp_table_cap(long long bytes);

/* Release the plan and its device memory (synchronises the device first). */
void dgt_plan_destroy(dgt_plan_t plan);

/* Human-readable status name, and the message of the last error on this host thread. */
const char* dgt_strerror(int status);
const char* dgt_last_error(void);

/* Per-kernel timing of the hot path.  dgt_profile_start() makes every later analysis,
 * synthesis and gradient call record a CUDA event pair on its stream around each kernel
 * launch; dgt_profile_stop() synchronises the device, writes a JSON object
 * {"kernel": {"launches": n, "ms": total}, ...} into json (cap bytes, NUL-terminated)
 * and turns recording off.  Not thread-safe; for measurement only. */
int dgt_profile_start(void);
int dgt_profile_stop(char* json, size_t cap);

/* Arithmetic throughput probe for roofline statements (no counterpart in the paper): runs
 * independent fused multiply-add chains on every SM of the current device and returns the
 * achieved rate in flop/s (2 per FMA per lane): kind 0 scalar float FMA, 1 packed float-pair
 * FMA, 2 double FMA.  Synchronises `stream`; allocates 4 bytes. */
int dgt_fma_rate(int kind, double* flops_per_s, void* stream);

/* Building block check: `howmany` contiguous complex transforms of length n (device buffers),
 * direction -1 (forward) or +1 (unnormalised inverse), precision DGT_F32 / DGT_F64. */
int dgt_fft_selftest(int64_t n, int precision, int direction, const void* in, void* out, int64_t howmany,
                     void* stream);

/* Bounds checking (no counterpart in the paper; a checking aid, not a step of the method).
 * A library compiled with -DDGT_DEBUG (libdgt_debug.so, selected in Python by DGT_DEBUG=1)
 * surrounds every device allocation it makes with 4096-byte guard zones of 0xFF bytes (a NaN
 * in float32 and float64), puts such zones between the regions of each analysis / synthesis
 * workspace (the plan's or the caller's, whose dgt_workspace_bytes grows accordingly), and
 * after every kernel launch checks every zone on the launching stream: an overwritten word
 * counts as a violation and is restored; nothing traps.  Out-of-bounds reads of a zone load
 * NaNs into the results.  That build serialises analysis / synthesis calls, synchronises the
 * device at the end of each and must not be captured into a CUDA graph; the caller's own
 * input and output buffers are not guarded.
 *
 * dgt_debug_build: 1 in the DGT_DEBUG build, else 0.
 * dgt_debug_status: synchronises the device; *violations = guard words found overwritten
 * since the previous call (then cleared); for the first of them, kernel (kernel_len bytes,
 * NUL-terminated; may be NULL) receives the name of the launch after which it was found and
 * *zone_offset its byte offset inside its guard zone (-1 when there is none).  Returns
 * DGT_ERR_UNSUPPORTED in the release build (nothing is checked there).
 * dgt_debug_touch_guard: overwrites the first word of the trailing guard zone of one of the
 * plan's allocations (memory the library owns), so that a test can see the next launch's
 * check report it.  DGT_ERR_UNSUPPORTED in the release build. */
int dgt_debug_build(void);
int dgt_debug_status(unsigned long long* violations, long long* zone_offset, char* kernel, size_t kernel_len);
int dgt_debug_touch_guard(dgt_plan_t plan);

#ifdef __cplusplus
}
#endif

#endif /* DGT_H */
