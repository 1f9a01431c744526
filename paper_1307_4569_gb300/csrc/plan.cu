// Host side of the library: lattice algebra, route selection, tables, device buffers, the
// orchestration of the kernels, and the extern "C" entry points declared in include/dgt.h.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/dgt.h"
#include "debug.h"
#include "engine.h"

using namespace dgt;

// ---------------------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------------------
static thread_local std::string g_last_error;

static int fail(int status, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return status;
}

namespace dgt {
long long g_wait_limit_cycles = kWaitCycles;
long long g_chirp_cap = 1ll << 30;     // bytes of chirp tables a plan created later may hold
}

#define CUDA_TRY(...)                                                                                 \
    do {                                                                                              \
        cudaError_t _e = (__VA_ARGS__);                                                                      \
        if (_e != cudaSuccess) {                                                                      \
            if (_e == cudaErrorMemoryAllocation) return fail(DGT_ERR_OOM, "%s: %s", #__VA_ARGS__, cudaGetErrorString(_e)); \
            return fail(DGT_ERR_CUDA, "%s: %s (%s:%d)", #__VA_ARGS__, cudaGetErrorString(_e), __FILE__, __LINE__);      \
        }                                                                                             \
    } while (0)

#define DGT_TRY(...)               \
    do {                           \
        int _s = (__VA_ARGS__);           \
        if (_s != DGT_OK) return _s; \
    } while (0)

// ---------------------------------------------------------------------------------------
// optional per-kernel timing: CUDA events recorded on the launching stream around every
// hot-path launch while profiling is on (dgt_profile_start / dgt_profile_stop)
// ---------------------------------------------------------------------------------------
struct ProfRec {
    const char* name;
    cudaEvent_t a, b;
};
static bool g_prof_on = false;
static std::vector<ProfRec> g_prof;
static std::vector<cudaEvent_t> g_prof_pool;
static size_t g_prof_used = 0;

static cudaEvent_t prof_event() {
    if (g_prof_used == g_prof_pool.size()) {
        cudaEvent_t e;
        cudaEventCreate(&e);
        g_prof_pool.push_back(e);
    }
    return g_prof_pool[g_prof_used++];
}

#define KTRY(NAME, ST, ...)                                           \
    do {                                                              \
        cudaEvent_t _ka = nullptr, _kb = nullptr;                     \
        if (g_prof_on) {                                              \
            _ka = prof_event();                                       \
            _kb = prof_event();                                       \
            cudaEventRecord(_ka, ST);                                 \
        }                                                             \
        CUDA_TRY(__VA_ARGS__);                                        \
        if (kDebug) dbg_after_launch(NAME, ST);                       \
        if (g_prof_on) {                                              \
            cudaEventRecord(_kb, ST);                                 \
            g_prof.push_back({NAME, _ka, _kb});                       \
        }                                                             \
    } while (0)

// ---------------------------------------------------------------------------------------
// integer lattice algebra (exact, int64)
// ---------------------------------------------------------------------------------------
static int64_t igcd(int64_t x, int64_t y) {
    x = x < 0 ? -x : x;
    y = y < 0 ? -y : y;
    while (y) {
        int64_t t = x % y;
        x = y;
        y = t;
    }
    return x;
}
static int64_t ilcm(int64_t x, int64_t y) { return x / igcd(x, y) * y; }
static int64_t pmod(int64_t x, int64_t m) {
    int64_t r = x % m;
    return r < 0 ? r + m : r;
}
// returns g = gcd(x, y) >= 0 and u, v with u x + v y = g
static int64_t egcd(int64_t x, int64_t y, int64_t& u, int64_t& v) {
    int64_t r0 = x, r1 = y, u0 = 1, u1 = 0, v0 = 0, v1 = 1;
    while (r1 != 0) {
        const int64_t qq = r0 / r1;
        int64_t t = r0 - qq * r1; r0 = r1; r1 = t;
        t = u0 - qq * u1; u0 = u1; u1 = t;
        t = v0 - qq * v1; v0 = v1; v1 = t;
    }
    if (r0 < 0) { r0 = -r0; u0 = -u0; v0 = -v0; }
    u = u0;
    v = v0;
    return r0;
}
// smallest x >= 0 with A x = B (mod m), or -1
static int64_t solve_congruence(int64_t A, int64_t B, int64_t m) {
    A = pmod(A, m);
    B = pmod(B, m);
    int64_t u, v;
    const int64_t g = egcd(A, m, u, v);
    if (B % g) return -1;
    const int64_t m2 = m / g;
    if (m2 == 1) return 0;
    const __int128 x = (__int128)(B / g) * (__int128)pmod(u, m2);
    return (int64_t)(x % m2);
}

struct ShearSel {
    int64_t s0, s1, b_r;
};

// Shear parameters with U_{s0,s1}^{-1} A separable (Theorem shearform).  A time shear alone
// (s0 = 0) works iff  s + k b = 0 (mod a)  has a solution k (proof of Prop. noshearlength):
// then s1 = -(s + k b)/a and the separable lattice is (a, b).  Otherwise the smallest s1 >= 0
// is taken for which eq. (modcond)  s0 X + a k1 = 0 (mod a b / X)  is solvable, with
// X = gcd(s1 a + s, b) = k1 (s1 a + s) + k2 b; the separable lattice is diag(a b / X, X).
// Every valid pair gives the same coefficients; among the frequency shears the first one in
// that order whose separable lattice this build can transform is taken (`runs`, given b_r = X),
// so that a lattice is refused only when none of them fits.
static bool shear_select(int64_t L, int64_t a, int64_t b, int64_t s, ShearSel& out,
                         const std::function<bool(int64_t)>& runs) {
    if (s == 0) {
        out = {0, 0, b};
        return true;
    }
    const int64_t k = solve_congruence(b, -s, a);
    if (k >= 0) {
        const int64_t num = s + k * b;          // divisible by a
        out = {0, pmod(-(num / a), L), b};
        return true;
    }
    bool found = false;
    for (int64_t s1 = 0; s1 < L; ++s1) {
        int64_t k1, k2;
        const int64_t X = egcd(s1 * a + s, b, k1, k2);
        const int64_t mod = a * b / X;
        const int64_t s0 = solve_congruence(X, -a * k1, mod);
        if (s0 >= 0) {
            if (!found) {
                out = {pmod(s0, L), s1, X};
                found = true;
            }
            if (runs(X)) {
                out = {pmod(s0, L), s1, X};
                return true;
            }
        }
    }
    return found;
}

// ---------------------------------------------------------------------------------------
// FFT plans and phase tables
// ---------------------------------------------------------------------------------------
static bool radix_plan(int64_t n, FftPlanDev& pl) {
    pl.n = (int)n;
    pl.nst = 0;
    int e2 = 0;
    int64_t m = n;
    while (m % 2 == 0) { m /= 2; ++e2; }
    std::vector<int> r;
    while (e2 >= 4 && e2 != 5) { r.push_back(16); e2 -= 4; }
    if (e2 == 5) { r.push_back(8); r.push_back(4); }
    else if (e2 == 3) r.push_back(8);
    else if (e2 == 2) r.push_back(4);
    else if (e2 == 1) r.push_back(2);
    for (int p : {3, 5, 7})
        while (m % p == 0) { r.push_back(p); m /= p; }
    if (m != 1 || (int)r.size() > kMaxStages) return false;
    for (size_t i = 0; i < r.size(); ++i) pl.R[i] = r[i];
    pl.nst = (int)r.size();
    return true;
}

// exp(2 pi i num / den) in double, reduced to an angle of modulus <= pi
static void cis_host(int64_t num, int64_t den, double& c, double& s) {
    int64_t r = pmod(num, den);
    if (2 * r > den) r -= den;
    const double ang = 2.0 * M_PI * (double)r / (double)den;
    c = std::cos(ang);
    s = std::sin(ang);
}

// FFT twiddles of length n: exp(-2 pi i e / n) for e < n; for a power of two n they are
// followed by the compact per-stage tables of the power-of-two kernels (fft_p2.cuh):
// entry n + s + k = exp(-2 pi i k / (16 s)) for s = 16^S with 16 s < n and k < s.
static std::vector<double> twiddle_host(int64_t n) {
    const bool p2 = n >= 16 && (n & (n - 1)) == 0;
    std::vector<double> h(2 * (size_t)(p2 ? 2 * n : n), 0.0);
    for (int64_t e = 0; e < n; ++e) cis_host(-e, n, h[2 * e], h[2 * e + 1]);
    if (p2)
        for (int64_t s = 16; 16 * s < n; s *= 16)
            for (int64_t k = 0; k < s; ++k) cis_host(-k, 16 * s, h[2 * (n + s + k)], h[2 * (n + s + k) + 1]);
    return h;
}

// the 16384-point float row transform of the power-of-two kernels (beyond the generic tile)
static bool row_only_len_ok(int64_t n, int precision) { return precision == DGT_F32 && n == 16384; }

struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf&) = delete;
    DevBuf& operator=(const DevBuf&) = delete;
    ~DevBuf() { dbg_free(p); }
    int alloc(size_t n) {
        if (n <= bytes && p) return DGT_OK;
        if (p) { dbg_free(p); p = nullptr; bytes = 0; }
        if (n == 0) return DGT_OK;
        cudaError_t e = dbg_malloc(&p, n);
        if (e != cudaSuccess) {
            cudaGetLastError();
            p = nullptr;
            return fail(DGT_ERR_OOM, "cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
        }
        bytes = n;
        return DGT_OK;
    }
};

template <typename T> static int upload_cplx(DevBuf& buf, const std::vector<double>& re_im, cudaStream_t st) {
    const size_t n = re_im.size() / 2;
    std::vector<T> h(2 * n);
    for (size_t i = 0; i < 2 * n; ++i) h[i] = (T)re_im[i];
    DGT_TRY(buf.alloc(sizeof(T) * 2 * n));
    CUDA_TRY(cudaMemcpyAsync(buf.p, h.data(), sizeof(T) * 2 * n, cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return DGT_OK;
}

template <typename T> struct TwTable {
    FftRef ref;
    DevBuf buf;
};

template <typename T> struct CisBuf {
    DevBuf hi, lo;
    CisTable<cplx<T>> tab;
};

template <typename T> static int make_cis(CisBuf<T>& cb, int64_t den, cudaStream_t st) {
    int shift = 0;
    while (((int64_t)1 << shift) * ((int64_t)1 << shift) < den) ++shift;
    const int64_t S = (int64_t)1 << shift;
    const int64_t nhi = den / S + 1;
    std::vector<double> hi(2 * nhi), lo(2 * S);
    for (int64_t k = 0; k < nhi; ++k) cis_host(k * S, den, hi[2 * k], hi[2 * k + 1]);
    for (int64_t r = 0; r < S; ++r) cis_host(r, den, lo[2 * r], lo[2 * r + 1]);
    DGT_TRY(upload_cplx<T>(cb.hi, hi, st));
    DGT_TRY(upload_cplx<T>(cb.lo, lo, st));
    cb.tab.hi = (const cplx<T>*)cb.hi.p;
    cb.tab.lo = (const cplx<T>*)cb.lo.p;
    cb.tab.md = make_mod((uint64_t)den);
    cb.tab.shift = shift;
    return DGT_OK;
}

// ---------------------------------------------------------------------------------------
// expiry words of the bounded device waits: one host-mapped word per plan, handed out from
// pinned pages that live until the process exits (so destroying a plan frees no pinned
// memory); the synthesis kernels write 1 into the word of the plan they run for
// ---------------------------------------------------------------------------------------
static std::mutex g_expiry_mu;
static std::vector<unsigned int*> g_expiry_free;
static std::vector<unsigned int*> g_expiry_live;

static int expiry_word_take(unsigned int** out) {
    std::lock_guard<std::mutex> lock(g_expiry_mu);
    if (g_expiry_free.empty()) {
        constexpr size_t kWords = 1024;
        void* page = nullptr;
        CUDA_TRY(cudaHostAlloc(&page, kWords * sizeof(unsigned int), cudaHostAllocMapped | cudaHostAllocPortable));
        unsigned int* w = (unsigned int*)page;
        for (size_t i = 0; i < kWords; ++i) {
            w[i] = 0;
            g_expiry_free.push_back(w + i);
        }
    }
    *out = g_expiry_free.back();
    g_expiry_free.pop_back();
    **out = 0;
    g_expiry_live.push_back(*out);
    return DGT_OK;
}
static void expiry_word_give(unsigned int* w) {
    if (!w) return;
    std::lock_guard<std::mutex> lock(g_expiry_mu);
    g_expiry_live.erase(std::remove(g_expiry_live.begin(), g_expiry_live.end(), w), g_expiry_live.end());
    g_expiry_free.push_back(w);
}
// read and clear a word (host side; the word is written by kernels through its mapping)
static unsigned int expiry_word_take_value(unsigned int* w) {
    if (!w) return 0;
    volatile unsigned int* v = w;
    const unsigned int x = *v;
    if (x) *v = 0;
    return x;
}

// the first bytes of a caller workspace hold its expiry word; the plan's work area follows
constexpr size_t kWsHeader = 256;

// ---------------------------------------------------------------------------------------
// the plan
// ---------------------------------------------------------------------------------------
struct PlanCore {
    int64_t L, a, M, lam1, lam2, b, N, s;
    int route, precision;
    int win_kind;
    int64_t Lg, center;
    int win_real;
    ShearSel sh{0, 0, 0};
    bool freq_shear = false;
    SepGeom sep{};
    int64_t J = 1;
    // Algorithm 1 constants (frequency-shear branch)
    int64_t ar = 0, Mr = 0, Nr = 0, C1 = 0, C2 = 0, C3m = 0, C4m = 0, C5m = 0, C6 = 0;
    int64_t L1 = 0, L2 = 0;            // FFT_L split
    int64_t fir_cols = 0, fir_group = 1;
    bool fir_synth_ok = true;
    bool fir_p2_synth = false;         // the FIR synthesis runs the power-of-two kernel
    std::vector<double> g_host;        // window as given (complex interleaved, float64)
    SepGeom coset_sep{};               // (lam2 a, M): used by the dual / tight Gram blocks
    int64_t ola_block = 0, ola_len = 0;  // blockwise plans: block length and local length
    int device = -1;                   // the CUDA device current at creation (owns the plan's memory)
};

// Streams, events and device staging slots of the host-buffer entry points (dgt_exec_host,
// idgt_exec_host), created on first use
struct HostPipe {
    cudaStream_t in = nullptr, out = nullptr;
    cudaEvent_t start = nullptr, last = nullptr, done_in[2] = {}, done_exec[2] = {}, done_out[2] = {};
    DevBuf src[2], dst[2];
    HostPipe() = default;
    HostPipe(const HostPipe&) = delete;
    HostPipe& operator=(const HostPipe&) = delete;
    ~HostPipe() {
        for (cudaEvent_t* e : {&start, &last, &done_in[0], &done_in[1], &done_exec[0], &done_exec[1], &done_out[0],
                               &done_out[1]})
            if (*e) cudaEventDestroy(*e);
        if (in) cudaStreamDestroy(in);
        if (out) cudaStreamDestroy(out);
    }
    int init() {
        if (in) return DGT_OK;
        CUDA_TRY(cudaStreamCreateWithFlags(&in, cudaStreamNonBlocking));
        CUDA_TRY(cudaStreamCreateWithFlags(&out, cudaStreamNonBlocking));
        for (cudaEvent_t* e : {&start, &last, &done_in[0], &done_in[1], &done_exec[0], &done_exec[1], &done_out[0],
                               &done_out[1]})
            CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
        return DGT_OK;
    }
};

struct dgt_plan_s {
    virtual ~dgt_plan_s() { expiry_word_give(expired); }
    std::unique_ptr<HostPipe> host_pipe;   // host-buffer entry points
    PlanCore core;
    unsigned int* expired = nullptr;   // host-mapped expiry word of the calls without a caller workspace
    virtual int exec(const void* f, int f_real, void* c, int64_t B, void* ws, cudaStream_t st) = 0;
    // `expired`: the word the synthesis kernels set when a bounded wait expires
    virtual int iexec(const void* c, void* f, int f_real, int64_t B, int which, void* ws, unsigned int* expired,
                      cudaStream_t st) = 0;
    virtual int window_out(int which, void* out, cudaStream_t st) = 0;
    virtual int iexec_window(const void* c, void* f, int f_real, int64_t B, const void* gamma, int gamma_real,
                             cudaStream_t st) {
        return fail(DGT_ERR_UNSUPPORTED, "synthesis with a caller's window is not available for this plan kind");
    }
    virtual int set_window(const void* g, int is_real, cudaStream_t st) = 0;
    virtual int grad_window(const void* f, int f_real, const void* G, void* grad, int grad_real, int64_t B,
                            cudaStream_t st) = 0;
    virtual int logmag(const void* c, void* G, double* loss, double eps, int64_t B, cudaStream_t st) = 0;
    virtual int fir_synthesis_noalloc(const void* c, void* f, int f_real, int64_t B, int which, cudaStream_t st) = 0;
    // DGT_DEBUG build: damage the trailing guard zone of one of the plan's allocations
    virtual int debug_touch_guard() { return DGT_ERR_UNSUPPORTED; }
    // synchronise st; a pending CUDA error, or an expired wait of this plan's own calls
    int status_check(cudaStream_t st) {
        CUDA_TRY(cudaStreamSynchronize(st));
        CUDA_TRY(cudaGetLastError());
        return pending_expiry();
    }
    // an expiry recorded by earlier work of this plan (no synchronisation: reported at the
    // next call once the kernel's write has landed); clears the word
    int pending_expiry() {
        if (expiry_word_take_value(expired))
            return fail(DGT_ERR_TIMEOUT, "a synthesis kernel of this plan gave up waiting for its tile copies");
        return DGT_OK;
    }
    virtual size_t ws_bytes(int64_t B) const = 0;
    virtual size_t owned_bytes() const = 0;
    // real-signal analysis / synthesis on channels 0..M/2 (through a plan-owned full array)
    virtual int exec_real(const void* f, void* ch, int64_t B, cudaStream_t st) = 0;
    virtual int iexec_real(const void* ch, void* f, int64_t B, int which, cudaStream_t st) = 0;
    DevBuf real_full;                  // staging for the real-signal entry points
};

// the real-signal symmetry holds for a real window, lambda2 <= 2 and an even M
static int real_ok(const PlanCore& k) {
    if (k.lam2 > 2 || k.M % 2) return fail(DGT_ERR_UNSUPPORTED, "real-signal coefficients need lambda2 <= 2 and an even M");
    if (!k.win_real) return fail(DGT_ERR_UNSUPPORTED, "real-signal coefficients need a real window");
    return DGT_OK;
}
template <typename T> static int exec_real_via(dgt_plan_s* p, const void* f, void* ch, int64_t B, cudaStream_t st) {
    const PlanCore& k = p->core;
    DGT_TRY(real_ok(k));
    if (B <= 0) return B == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
    DGT_TRY(p->real_full.alloc(sizeof(cplx<T>) * (size_t)B * k.N * k.M));
    DGT_TRY(p->exec(f, 1, p->real_full.p, B, nullptr, st));
    KTRY("half_compact", st, launch_half_compact<T>((const cplx<T>*)p->real_full.p, (cplx<T>*)ch, k.N, k.M, B, st));
    return DGT_OK;
}
template <typename T>
static int iexec_real_via(dgt_plan_s* p, const void* ch, void* f, int64_t B, int which, cudaStream_t st) {
    const PlanCore& k = p->core;
    DGT_TRY(real_ok(k));
    if (B <= 0) return B == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
    DGT_TRY(p->real_full.alloc(sizeof(cplx<T>) * (size_t)B * k.N * k.M));
    KTRY("half_expand", st, launch_half_expand<T>((const cplx<T>*)ch, (cplx<T>*)p->real_full.p, k.N, k.M, k.lam1, k.lam2,
                                                  B, st));
    return p->iexec(p->real_full.p, f, 1, B, which, nullptr, p->expired, st);
}

template <typename T> struct PlanImpl final : dgt_plan_s {
    using C = cplx<T>;
    std::map<int64_t, std::unique_ptr<TwTable<T>>> tw;      // FFT length -> table
    CisBuf<T> cisL, cis2L, cis2N, cisLM;
    DevBuf sigma;                      // coset shifts (int64, J)
    DevBuf g64;                        // window, float64 complex (L, or Lg taps for FIR)
    DevBuf gT;                         // window in T (L or Lg)
    DevBuf zg[4];                      // window factors: 0 analysis/adjoint, 1 dual, 2 tight, 3 caller's
    bool zg_ok[4] = {false, false, false, false};
    DevBuf gam[4];                     // gamma in T (full length L, or Lg taps for FIR)
    DevBuf work;                       // plan-owned workspace
    DevBuf tmpwin;                     // scratch for window set-up
    DevBuf status;                     // int flag for the Gram solve
    DevBuf firmt[4];                   // FIR route: modulated taps [lam2][Lg] of the windows in gam / gT
    DevBuf lossparts;
    DevBuf hbtab;                      // FIR route, lambda2 = 2: exp(-pi i k / M), k < M (real-input pairing)
    std::map<int64_t, DevBuf> chirpt;  // shear routes: s mod 2L -> pchirp(L, s)(l), l < L

    int debug_touch_guard() override {
        return sigma.p ? dbg_touch_trailing_guard(sigma.p, sigma.bytes) : DGT_ERR_UNSUPPORTED;
    }
    DevBuf gradws;                     // work arrays of the window gradient

    const FftRef* fft(int64_t n) {
        auto it = tw.find(n);
        return it == tw.end() ? nullptr : &it->second->ref;
    }
    // rows: the length is only used by the row kernels (fft_post / pre_ifft), which also have
    // a 16384-point float path beyond the generic shared-memory tile
    int add_fft(int64_t n, cudaStream_t st, bool rows = false) {
        if (tw.count(n)) return DGT_OK;
        auto t = std::make_unique<TwTable<T>>();
        if (!radix_plan(n, t->ref.pl))
            return fail(DGT_ERR_UNSUPPORTED, "FFT length %lld has a prime factor above 7", (long long)n);
        if (n + 1 > tile_cap<T>() && !(rows && row_only_len_ok(n, sizeof(T) == 4 ? DGT_F32 : DGT_F64)))
            return fail(DGT_ERR_UNSUPPORTED, "FFT length %lld exceeds the shared-memory tile (%lld)", (long long)n,
                        (long long)tile_cap<T>());
        DGT_TRY(upload_cplx<T>(t->buf, twiddle_host(n), st));
        t->ref.tw = t->buf.p;
        tw[n] = std::move(t);
        return DGT_OK;
    }

    // ---- workspace layout -----------------------------------------------------------
    // regions of the workspace; the DGT_DEBUG build puts a guard zone before, between and after
    // them (guard[0..ng)), checked after every launch of the call
    struct Layout {
        size_t zf, y, tmp, fh, seams, total;
        size_t guard[5];
        int ng;
    };
    static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
    Layout layout(int64_t B) const {
        const PlanCore& k = core;
        Layout ly{};
        size_t off = 0;
        auto gz = [&]() {
            if (kDebug) {
                ly.guard[ly.ng++] = off;
                off += kGuard;
            }
        };
        gz();
        if (k.route == DGT_ROUTE_FIR) {
            FirParams<C> fp{};
            fp.N = k.N; fp.cols = k.fir_cols; fp.Lg = k.Lg; fp.a = k.a;
            ly.seams = off;
            off += al(sizeof(C) * (size_t)B * fir_seam_elems(fp));
            gz();
            ly.total = off;
            return ly;
        }
        ly.zf = off;
        off += al(sizeof(C) * (size_t)B * k.L);
        gz();
        ly.y = off;
        off += al(sizeof(C) * (size_t)B * k.J * k.sep.d * k.sep.q * k.sep.M);
        gz();
        if (k.freq_shear) {
            ly.tmp = off;
            off += al(sizeof(C) * (size_t)B * k.L);
            gz();
            ly.fh = off;
            off += al(sizeof(C) * (size_t)B * k.L);
            gz();
        }
        ly.total = off;
        return ly;
    }
    size_t ws_bytes(int64_t B) const override { return layout(B).total; }
    size_t owned_bytes() const override {
        size_t s = sigma.bytes + g64.bytes + gT.bytes + work.bytes + tmpwin.bytes + status.bytes + lossparts.bytes +
                   real_full.bytes + hbtab.bytes + gradws.bytes;
        for (auto& kv : chirpt) s += kv.second.bytes;
        for (int i = 0; i < 4; ++i) s += zg[i].bytes + gam[i].bytes + firmt[i].bytes;
        for (auto& kv : tw) s += kv.second->buf.bytes;
        s += cisL.hi.bytes + cisL.lo.bytes + cis2L.hi.bytes + cis2L.lo.bytes + cis2N.hi.bytes + cis2N.lo.bytes +
             cisLM.hi.bytes + cisLM.lo.bytes;
        return s;
    }

    ChirpParams<C> chirp(int64_t s, int conj) const {
        ChirpParams<C> cp{};
        cp.mode = pmod(s, 2 * core.L) == 0 ? PRE_NONE : PRE_CHIRP;
        cp.L = core.L;
        cp.s_2L = pmod(s, 2 * core.L);
        cp.conj = conj;
        cp.cis2L = cis2L.tab;
        cp.m2L = make_mod(2 * (uint64_t)core.L);
        auto it = chirpt.find(cp.s_2L);
        cp.tab = it == chirpt.end() ? nullptr : (const C*)it->second.p;
        return cp;
    }
    // the chirps of Algorithm 1 (pchirp(L, s1), and pchirp(L, -s0) in the frequency-shear branch)
    // as tables of L values, so that a kernel reads each sample's factor in one load; none
    // beyond g_chirp_cap bytes per plan, where the kernels compute the factors
    int add_chirp(int64_t s, cudaStream_t st) {
        const ChirpParams<C> cp = chirp(s, 0);
        if (cp.mode != PRE_CHIRP || cp.tab) return DGT_OK;
        size_t have = 0;
        for (auto& kv : chirpt) have += kv.second.bytes;
        const size_t bytes = sizeof(C) * (size_t)core.L;
        if ((long long)(have + bytes) > g_chirp_cap) return DGT_OK;
        DevBuf& b = chirpt[cp.s_2L];
        DGT_TRY(b.alloc(bytes));
        KTRY("chirp_table", st, launch_chirp_table<T>(cp, (C*)b.p, st));
        return DGT_OK;
    }
    ChirpParams<C> nochirp() const {
        ChirpParams<C> cp{};
        cp.mode = PRE_NONE;
        cp.L = core.L;
        cp.cis2L = cis2L.tab;
        cp.m2L = make_mod(2 * (uint64_t)core.L);
        return cp;
    }

    PostParams<C> post() const {
        const PlanCore& k = core;
        PostParams<C> pp{};
        pp.L = k.L; pp.M = k.M; pp.N = k.N; pp.b = k.b; pp.a = k.a;
        pp.cisL = cisL.tab;
        pp.cis2N = cis2N.tab;
        pp.mL = make_mod((uint64_t)k.L);
        pp.mN = make_mod((uint64_t)k.N);
        pp.m2N = make_mod(2 * (uint64_t)k.N);
        pp.mb = make_mod((uint64_t)k.b);
        pp.lam1 = k.lam1;
        pp.lam2 = k.lam2;
        if (k.route == DGT_ROUTE_COSET) {
            pp.mode = POST_COSET;
            pp.lam2 = k.lam2;
            pp.at = k.lam2 * k.a;
            pp.sigma = (const int64_t*)sigma.p;
        } else if (!k.freq_shear) {
            pp.mode = POST_SHEAR0;
            pp.s1a_modL = (int64_t)(((__int128)k.sh.s1 * k.a) % k.L);
            pp.C1_2N = (int64_t)(((__int128)k.sh.s1 * k.a % (2 * k.N)) * ((k.L + 1) % (2 * k.N)) % (2 * k.N));
        } else {
            const int64_t twoN = 2 * k.N;
            pp.mode = POST_SHEAR1;
            pp.Nr = k.Nr;
            pp.C1 = k.C1;
            pp.C2_N = pmod(k.C2, k.N);
            pp.C1_2N_ = pmod(k.C1, twoN);
            pp.C2_2N = pmod(k.C2, twoN);
            pp.C3_2N = k.C3m;
            pp.C4_2N = k.C4m;
            pp.C5_2N = k.C5m;
            pp.s1ar_L = pmod(-(int64_t)(((__int128)k.sh.s1 * k.ar) % k.L), k.L);
            pp.C6_L = pmod(k.C6, k.L);
            // 32-bit per-row form when every product stays below 2^32
            if (twoN < 65536 && (uint64_t)k.L * (uint64_t)(k.Nr + 1) < ((uint64_t)1 << 32)) {
                pp.sh1_fast = 1;
                pp.f_Nr = (uint32_t)k.Nr; pp.f_N = (uint32_t)k.N; pp.f_M = (uint32_t)k.M;
                pp.f_C1 = (uint32_t)pp.C1_2N_; pp.f_C2 = (uint32_t)pp.C2_2N; pp.f_C3 = (uint32_t)pp.C3_2N;
                pp.f_C4 = (uint32_t)pp.C4_2N; pp.f_C5 = (uint32_t)pp.C5_2N;
                pp.f_s1ar = (uint32_t)pp.s1ar_L; pp.f_C6 = (uint32_t)pp.C6_L;
                pp.q2N = make_mod32((uint32_t)twoN);
                pp.qL = make_mod32((uint32_t)k.L);
                pp.qb = make_mod32((uint32_t)k.b);
            }
        }
        return pp;
    }

    // ---- set-up -----------------------------------------------------------------------
    int init(cudaStream_t st) {
        PlanCore& k = core;
        DGT_TRY(make_cis(cisL, k.L, st));
        DGT_TRY(make_cis(cis2L, 2 * k.L, st));
        DGT_TRY(make_cis(cis2N, 2 * k.N, st));
        DGT_TRY(make_cis(cisLM, k.lam2 * k.M, st));
        if (k.route == DGT_ROUTE_SHEAR) {
            DGT_TRY(add_chirp(k.sh.s1, st));
            if (k.freq_shear) DGT_TRY(add_chirp(-k.sh.s0, st));
        }
        // coset shifts sigma_j = j s mod b (Prop. mwindec)
        std::vector<int64_t> sg(k.lam2);
        for (int64_t j = 0; j < k.lam2; ++j) sg[j] = (j * k.s) % k.b;
        DGT_TRY(sigma.alloc(sizeof(int64_t) * k.lam2));
        CUDA_TRY(cudaMemcpyAsync(sigma.p, sg.data(), sizeof(int64_t) * k.lam2, cudaMemcpyHostToDevice, st));
        DGT_TRY(status.alloc(sizeof(int)));
        // FFT tables
        if (k.route == DGT_ROUTE_FIR) {
            DGT_TRY(add_fft(k.M, st));
            if (k.lam2 == 2) {
                std::vector<double> hb(2 * (size_t)k.M);
                for (int64_t e = 0; e < k.M; ++e) cis_host(-e, 2 * k.M, hb[2 * e], hb[2 * e + 1]);
                DGT_TRY(upload_cplx<T>(hbtab, hb, st));
            }
        } else {
            DGT_TRY(add_fft(k.sep.d, st));
            DGT_TRY(add_fft(k.sep.M, st, true));
            if (k.freq_shear) {
                DGT_TRY(add_fft(k.L1, st));
                DGT_TRY(add_fft(k.L2, st));
            }
        }
        // coset Gram lattice tables (dual / tight)
        DGT_TRY(add_fft_if_ok(k.coset_sep.d, st));
        // upload the window (float64)
        const int64_t n = (int64_t)k.g_host.size() / 2;
        std::vector<double> gh = k.g_host;
        DGT_TRY(upload_cplx<double>(g64, gh, st));
        DGT_TRY(gT.alloc(sizeof(C) * n));
        KTRY("convert", st, launch_convert<double, T>(g64.p, 0, (C*)gT.p, n, st));
        DGT_TRY(build_factor(0, (const C*)gT.p, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return DGT_OK;
    }
    int add_fft_if_ok(int64_t n, cudaStream_t st) {
        // the dual / tight set-up is optional: failures surface when it is requested
        FftPlanDev pl;
        if (!radix_plan(n, pl) || n + 1 > tile_cap<T>()) return DGT_OK;
        return add_fft(n, st);
    }

    // window factor of `gam` (device, T, full length L or FIR taps) into zg[slot]
    int build_factor(int slot, const C* gw, cudaStream_t st) {
        const PlanCore& k = core;
        if (k.route == DGT_ROUTE_FIR) {
            // FIR route: the taps themselves plus their modulated copies (slot 0 is built from
            // the float64 window g64, which holds the same taps)
            DGT_TRY(build_fir_mt(slot, (const double2*)g64.p, st));
            zg_ok[slot] = true;
            return DGT_OK;
        }
        DGT_TRY(zg[slot].alloc(sizeof(C) * (size_t)k.J * k.L));
        C* out = (C*)zg[slot].p;
        const FftRef* fd = fft(k.sep.d);
        if (k.route == DGT_ROUTE_COSET) {
            DGT_TRY(tmpwin.alloc(sizeof(C) * (size_t)k.J * k.L));
            KTRY("coset_windows", st, launch_coset_windows<T>(gw, (C*)tmpwin.p, k.L, k.a, k.J, (const int64_t*)sigma.p, cisL.tab, st));
            KTRY("zak_fwd", st, launch_zak_fwd<T>(tmpwin.p, 0, k.L, out, k.L, k.L, k.sep.d, *fd, nochirp(), k.J, st));
        } else if (!k.freq_shear) {
            KTRY("zak_fwd", st, launch_zak_fwd<T>(gw, 0, k.L, out, k.L, k.L, k.sep.d, *fd, chirp(k.sh.s1, 0), 1, st));
        } else {
            // g^ = pchirp(L, -s0) FFT(pchirp(L, s1) g) / L   (Algorithm 1, frequency-shear branch)
            DGT_TRY(tmpwin.alloc(sizeof(C) * 2 * (size_t)k.L));
            C* t1 = (C*)tmpwin.p;
            C* t2 = t1 + k.L;
            KTRY("fftL_cols", st, launch_fftL_cols<T>(gw, 0, t1, k.L1, k.L2, -1, *fft(k.L1), chirp(k.sh.s1, 0), cisL.tab, 1, st));
            KTRY("fftL_rows", st, launch_fftL_rows<T>(t1, t2, 0, k.L1, k.L2, -1, *fft(k.L2), chirp(-k.sh.s0, 0), (T)1 / (T)k.L, 1, st));
            KTRY("zak_fwd", st, launch_zak_fwd<T>(t2, 0, k.L, out, k.L, k.L, k.sep.d, *fd, nochirp(), 1, st));
        }
        zg_ok[slot] = true;
        return DGT_OK;
    }

    // [lam2][Lg] modulated taps, then the Lg real parts of row 0 (the taps themselves for a real
    // window) as a dense array for the paired kernels
    int build_fir_mt(int slot, const double2* taps64, cudaStream_t st) {
        const PlanCore& k = core;
        const size_t mt = sizeof(C) * (size_t)k.lam2 * k.Lg;
        DGT_TRY(firmt[slot].alloc(mt + sizeof(T) * (size_t)k.Lg));
        KTRY("fir_modtaps", st, launch_fir_modtaps<T>(taps64, (C*)firmt[slot].p, k.Lg, k.lam2, k.M, st));
        CUDA_TRY(cudaMemcpy2DAsync((char*)firmt[slot].p + mt, sizeof(T), firmt[slot].p, sizeof(C), sizeof(T),
                                   (size_t)k.Lg, cudaMemcpyDeviceToDevice, st));
        return DGT_OK;
    }

    int set_window(const void* g, int is_real, cudaStream_t st) override {
        const PlanCore& k = core;
        const int64_t n = k.win_kind == DGT_WINDOW_FIR ? k.Lg : k.L;
        KTRY("convert", st, launch_convert<T, T>(g, is_real, (C*)gT.p, n, st));
        KTRY("convert", st, launch_convert<T, double>(g, is_real, (double2*)g64.p, n, st));
        core.win_real = is_real;
        zg_ok[1] = zg_ok[2] = false;
        return build_factor(0, (const C*)gT.p, st);
    }

    // the power-of-two fused Zak kernels apply: p = 1 (so the Zak columns are the product
    // columns, K0 = M) and a power-of-two Zak length
    bool fused_zak() const {
        const SepGeom& g = core.sep;
        return g.p == 1 && g.K0 == g.M && p2_col_len_ok(g.d);
    }

    // ---- analysis ---------------------------------------------------------------------
    int exec(const void* f, int f_real, void* c, int64_t B, void* wsp, cudaStream_t st) override {
        return exec_core(f, f_real, c, B, wsp, st, false);
    }
    // half: the coefficients hold channels 0..M/2 only (real signals; half_io checked)
    int exec_core(const void* f, int f_real, void* c, int64_t B, void* wsp, cudaStream_t st, bool half) {
        const PlanCore& k = core;
        if (B <= 0) return B == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
        const Layout ly = layout(B);
        char* ws = (char*)wsp;
        if (!ws) {
            DGT_TRY(work.alloc(ly.total));
            ws = (char*)work.p;
        }
        DbgScope dbg(st, ws, ly.guard, ly.ng);
        if (k.route == DGT_ROUTE_FIR) {
            FirParams<C> fp = fir_params(0);
            fp.half = half;
            KTRY("fir_analysis", st, launch_fir_analysis<T>(f, f_real, (C*)c, fp, *fft(k.M), B, st));
            return DGT_OK;
        }
        C* zf = (C*)(ws + ly.zf);
        C* y = (C*)(ws + ly.y);
        const FftRef* fd = fft(k.sep.d);
        // the Zak input: the signal (coset: as it is; time shear: times pchirp(s1)), or its
        // chirped FFT_L (frequency shear)
        const void* zsrc = f;
        int zreal = f_real;
        ChirpParams<C> pre = k.route == DGT_ROUTE_COSET ? nochirp() : chirp(k.sh.s1, 0);
        if (k.freq_shear) {
            C* tmp = (C*)(ws + ly.tmp);
            C* fh = (C*)(ws + ly.fh);
            KTRY("fftL_cols", st, launch_fftL_cols<T>(f, f_real, tmp, k.L1, k.L2, -1, *fft(k.L1), chirp(k.sh.s1, 0), cisL.tab, B, st));
            KTRY("fftL_rows", st, launch_fftL_rows<T>(tmp, fh, 0, k.L1, k.L2, -1, *fft(k.L2), chirp(-k.sh.s0, 0), (T)1, B, st));
            zsrc = fh;
            zreal = 0;
            pre = nochirp();
        }
        if (fused_zak()) {
            KTRY("zak_prod_ifft", st, p2_zak_prod_ifft<T>(zsrc, zreal, k.L, (const C*)zg[0].p, k.J, y, k.sep, fd->tw, pre, B, st));
        } else {
            KTRY("zak_fwd", st, launch_zak_fwd<T>(zsrc, zreal, k.L, zf, k.L, k.L, k.sep.d, *fd, pre, B, st));
            KTRY("prod_ifft", st, launch_prod_ifft<T>(zf, (const C*)zg[0].p, k.J, y, k.sep, *fd, B, st));
        }
        PostParams<C> pp = post();
        pp.half = half;
        KTRY("fft_post", st, launch_fft_post<T>(y, (C*)c, k.sep, k.J, *fft(k.sep.M), pp, B, st));
        return DGT_OK;
    }

    // FIR parameters for window slot 0 (analysis / adjoint), 1 (dual) or 2 (tight)
    FirParams<C> fir_params(int which) const {
        const PlanCore& k = core;
        FirParams<C> fp{};
        fp.L = k.L; fp.a = k.a; fp.M = k.M; fp.N = k.N; fp.lam1 = k.lam1; fp.lam2 = k.lam2;
        fp.Lg = k.Lg; fp.center = k.center; fp.cisLM = cisLM.tab; fp.cols = k.fir_cols;
        fp.taps = which == 0 ? (const C*)gT.p : (const C*)gam[which].p;
        fp.mtaps = (const C*)firmt[which].p;
        fp.rtaps = firmt[which].p ? (const T*)((const char*)firmt[which].p + sizeof(C) * (size_t)k.lam2 * k.Lg)
                                  : nullptr;
        fp.mN = make_mod((uint64_t)k.N);
        fp.group = k.fir_group;
        fp.pairable = which <= 2 && k.win_real;
        fp.hb = (const C*)hbtab.p;
        return fp;
    }

    // ---- synthesis ----------------------------------------------------------------------
    int ensure_window(int which, cudaStream_t st) {
        if (which == 0 || zg_ok[which]) return DGT_OK;
        const PlanCore& k = core;
        const int tight = which == 2;
        if (k.route == DGT_ROUTE_FIR || k.win_kind == DGT_WINDOW_FIR) {
            if (k.Lg > k.M)
                return fail(DGT_ERR_UNSUPPORTED, "dual / tight of an FIR window longer than M is not implemented");
        }
        CUDA_TRY(cudaMemsetAsync(status.p, 0, sizeof(int), st));
        if (k.win_kind == DGT_WINDOW_FIR) {
            // short window: S is diagonal; gamma has the same support
            DevBuf g64o;
            DGT_TRY(g64o.alloc(sizeof(double2) * k.Lg));
            KTRY("fir_dual", st, launch_fir_dual((const double2*)g64.p, (double2*)g64o.p, k.Lg, k.a, k.M, tight, (int*)status.p, st));
            DGT_TRY(check_status(st));
            if (k.route == DGT_ROUTE_FIR) {
                DGT_TRY(gam[which].alloc(sizeof(C) * k.Lg));
                KTRY("convert", st, launch_convert<double, T>(g64o.p, 0, (C*)gam[which].p, k.Lg, st));
                DGT_TRY(build_fir_mt(which, (const double2*)g64o.p, st));
                zg_ok[which] = true;
                CUDA_TRY(cudaStreamSynchronize(st));
                return DGT_OK;
            }
            // Zak route with an FIR window: expand gamma to full length
            DevBuf full;
            DGT_TRY(full.alloc(sizeof(double2) * k.L));
            std::vector<double> taps(2 * k.Lg);
            CUDA_TRY(cudaMemcpyAsync(taps.data(), g64o.p, sizeof(double2) * k.Lg, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<double> fullh(2 * k.L, 0.0);
            for (int64_t t = 0; t < k.Lg; ++t) {
                const int64_t l = pmod(t - k.center, k.L);
                fullh[2 * l] = taps[2 * t];
                fullh[2 * l + 1] = taps[2 * t + 1];
            }
            DGT_TRY(upload_cplx<T>(gam[which], fullh, st));
            DGT_TRY(build_factor(which, (const C*)gam[which].p, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            return DGT_OK;
        }
        // full window: Zak-domain Gram blocks of the coset decomposition, float64
        const SepGeom& cg = k.coset_sep;
        if (cg.p > 8) return fail(DGT_ERR_UNSUPPORTED, "Gram blocks of size %lld > 8", (long long)cg.p);
        TwTable<double> twd;
        if (!radix_plan(cg.d, twd.ref.pl) || cg.d + 1 > tile_cap<double>())
            return fail(DGT_ERR_UNSUPPORTED, "dual window: Zak length %lld unsupported", (long long)cg.d);
        {
            DGT_TRY(upload_cplx<double>(twd.buf, twiddle_host(cg.d), st));
            twd.ref.tw = twd.buf.p;
        }
        CisBuf<double> cisL64;
        DGT_TRY(make_cis(cisL64, k.L, st));
        DevBuf gj, zj, zo, gout;
        DGT_TRY(gj.alloc(sizeof(double2) * (size_t)k.lam2 * k.L));
        DGT_TRY(zj.alloc(sizeof(double2) * (size_t)k.lam2 * k.L));
        DGT_TRY(zo.alloc(sizeof(double2) * (size_t)k.L));
        DGT_TRY(gout.alloc(sizeof(double2) * (size_t)k.L));
        KTRY("coset_windows", st, launch_coset_windows<double>((const double2*)g64.p, (double2*)gj.p, k.L, k.a, k.lam2,
                                              (const int64_t*)sigma.p, cisL64.tab, st));
        ChirpParams<double2> none{};
        none.mode = PRE_NONE;
        none.L = k.L;
        KTRY("zak_fwd", st, launch_zak_fwd<double>(gj.p, 0, k.L, (double2*)zj.p, k.L, k.L, cg.d, twd.ref, none, k.lam2, st));
        KTRY("gram_solve", st, launch_gram_solve((const double2*)zj.p, k.lam2, (double2*)zo.p, cg, tight, (int*)status.p, st));
        DGT_TRY(check_status(st));
        KTRY("zak_inv", st, launch_zak_inv<double>((const double2*)zo.p, k.L, gout.p, 0, k.L, k.L, cg.d, twd.ref, none,
                                        1.0 / (double)cg.d, 1, st));
        DGT_TRY(gam[which].alloc(sizeof(C) * k.L));
        KTRY("convert", st, launch_convert<double, T>(gout.p, 0, (C*)gam[which].p, k.L, st));
        DGT_TRY(build_factor(which, (const C*)gam[which].p, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return DGT_OK;
    }
    int check_status(cudaStream_t st) {
        int h = 0;
        CUDA_TRY(cudaMemcpyAsync(&h, status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        if (h) return fail(DGT_ERR_NOT_FRAME, "a Gram block is singular or ill-conditioned: no frame");
        return DGT_OK;
    }

    int iexec(const void* c, void* f, int f_real, int64_t B, int which, void* wsp, unsigned int* expired,
              cudaStream_t st) override {
        return iexec_core(c, f, f_real, B, which, wsp, expired, st, false);
    }
    // synthesis with the caller's window (slot 3): its factorisation is built on `st` first
    int iexec_window(const void* c, void* f, int f_real, int64_t B, const void* gamma, int gamma_real,
                     cudaStream_t st) override {
        const PlanCore& k = core;
        if (B <= 0) return B == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
        const bool fir = k.route == DGT_ROUTE_FIR;
        const int64_t n = fir ? k.Lg : k.L;
        zg_ok[3] = false;
        DGT_TRY(gam[3].alloc(sizeof(C) * n));
        KTRY("convert", st, launch_convert<T, T>(gamma, gamma_real, (C*)gam[3].p, n, st));
        if (fir) {
            DGT_TRY(tmpwin.alloc(sizeof(double2) * n));
            KTRY("convert", st, launch_convert<T, double>(gamma, gamma_real, (double2*)tmpwin.p, n, st));
            DGT_TRY(build_fir_mt(3, (const double2*)tmpwin.p, st));
            zg_ok[3] = true;
        } else {
            DGT_TRY(build_factor(3, (const C*)gam[3].p, st));
        }
        return iexec_core(c, f, f_real, B, 3, nullptr, expired, st, false);
    }
    int iexec_core(const void* c, void* f, int f_real, int64_t B, int which, void* wsp, unsigned int* expired,
                   cudaStream_t st, bool half) {
        const PlanCore& k = core;
        if (which < 0 || which > 3) return fail(DGT_ERR_ARG, "bad synthesis window %d", which);
        if (B <= 0) return B == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
        if (!zg_ok[which]) {
            if (wsp) return fail(DGT_ERR_ARG, "the dual / tight window is not cached yet (call dgt_window_dual/_tight)");
            DGT_TRY(ensure_window(which, st));
        }
        const Layout ly = layout(B);
        char* ws = (char*)wsp;
        if (!ws) {
            DGT_TRY(work.alloc(ly.total));
            ws = (char*)work.p;
        }
        DbgScope dbg(st, ws, ly.guard, ly.ng);
        if (k.route == DGT_ROUTE_FIR) {
            if (!k.fir_synth_ok)
                return fail(DGT_ERR_UNSUPPORTED, "FIR synthesis: %lld columns per tile cannot cover a window of %lld",
                            (long long)k.fir_cols, (long long)k.Lg);
            FirParams<C> fp = fir_params(which);
            fp.half = half;
            KTRY("fir_synthesis", st, launch_fir_synthesis<T>((const C*)c, f, f_real, (C*)(ws + ly.seams), fp, *fft(k.M), B, st));
            return DGT_OK;
        }
        C* zf = (C*)(ws + ly.zf);
        C* y = (C*)(ws + ly.y);
        const FftRef* fd = fft(k.sep.d);
        PostParams<C> ppi = post();
        ppi.half = half;
        KTRY("pre_ifft", st, launch_pre_ifft<T>((const C*)c, y, k.sep, k.J, *fft(k.sep.M), ppi, B, st));
        KTRY("fft_prod_adj", st, launch_fft_prod_adj<T>(y, (const C*)zg[which].p, k.J, zf, k.sep, *fd, B, expired, st));
        if (k.route == DGT_ROUTE_COSET) {
            KTRY("zak_inv", st, launch_zak_inv<T>(zf, k.L, f, f_real, k.L, k.L, k.sep.d, *fd, nochirp(), (T)1, B, st));
        } else if (!k.freq_shear) {
            KTRY("zak_inv", st, launch_zak_inv<T>(zf, k.L, f, f_real, k.L, k.L, k.sep.d, *fd, chirp(k.sh.s1, 1), (T)1, B, st));
        } else {
            C* tmp = (C*)(ws + ly.tmp);
            C* fh = (C*)(ws + ly.fh);
            KTRY("zak_inv", st, launch_zak_inv<T>(zf, k.L, fh, 0, k.L, k.L, k.sep.d, *fd, nochirp(), (T)1, B, st));
            // adjoint of f -> pchirp(-s0) FFT(pchirp(s1) f): conj chirps, unnormalised inverse DFT
            KTRY("fftL_cols", st, launch_fftL_cols<T>(fh, 0, tmp, k.L1, k.L2, +1, *fft(k.L1), chirp(-k.sh.s0, 1), cisL.tab, B, st));
            KTRY("fftL_rows", st, launch_fftL_rows<T>(tmp, f, f_real, k.L1, k.L2, +1, *fft(k.L2), chirp(k.sh.s1, 1), (T)1, B, st));
        }
        return DGT_OK;
    }

    int window_out(int which, void* out, cudaStream_t st) override {
        const PlanCore& k = core;
        DGT_TRY(ensure_window(which, st));
        if (k.route == DGT_ROUTE_FIR) {
            // expand the taps to a full-length window
            std::vector<T> taps(2 * k.Lg);
            CUDA_TRY(cudaMemcpyAsync(taps.data(), gam[which].p, sizeof(C) * k.Lg, cudaMemcpyDeviceToHost, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            std::vector<T> full(2 * k.L, (T)0);
            for (int64_t t = 0; t < k.Lg; ++t) {
                const int64_t l = pmod(t - k.center, k.L);
                full[2 * l] = taps[2 * t];
                full[2 * l + 1] = taps[2 * t + 1];
            }
            CUDA_TRY(cudaMemcpyAsync(out, full.data(), sizeof(C) * k.L, cudaMemcpyHostToDevice, st));
            CUDA_TRY(cudaStreamSynchronize(st));
            return DGT_OK;
        }
        CUDA_TRY(cudaMemcpyAsync(out, gam[which].p, sizeof(C) * k.L, cudaMemcpyDeviceToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return DGT_OK;
    }

    // ---- gradients ------------------------------------------------------------------------
    int grad_window(const void* f, int f_real, const void* G, void* grad, int grad_real, int64_t B,
                    cudaStream_t st) override {
        const PlanCore& k = core;
        if (k.win_kind != DGT_WINDOW_FULL) return fail(DGT_ERR_UNSUPPORTED, "window gradient needs a full-length window");
        // through the coset decomposition (any route gives the same coefficients)
        const SepGeom& cg = k.coset_sep;
        DGT_TRY(add_fft(cg.d, st));
        DGT_TRY(add_fft(cg.M, st, true));
        const FftRef* fd = fft(cg.d);
        PostParams<C> pp{};
        pp.mode = POST_COSET;
        pp.L = k.L; pp.M = k.M; pp.N = k.N; pp.b = k.b; pp.a = k.a;
        pp.lam2 = k.lam2; pp.at = k.lam2 * k.a; pp.sigma = (const int64_t*)sigma.p;
        pp.cisL = cisL.tab; pp.cis2N = cis2N.tab;
        pp.mL = make_mod((uint64_t)k.L);
        pp.mN = make_mod((uint64_t)k.N);
        pp.m2N = make_mod(2 * (uint64_t)k.N);
        pp.mb = make_mod((uint64_t)k.b);
        const int64_t groups = fft_grad_window_groups(cg, k.lam2, B, sizeof(C));
        const size_t need = al(sizeof(C) * (size_t)B * k.L) + al(sizeof(C) * (size_t)B * k.M * k.N) +
                            2 * al(sizeof(C) * (size_t)k.lam2 * k.L) + al(sizeof(C) * (size_t)groups * k.lam2 * k.L);
        DGT_TRY(gradws.alloc(need));               // plan-owned, grown on demand
        char* p = (char*)gradws.p;
        C* zf = (C*)p; p += al(sizeof(C) * (size_t)B * k.L);
        C* y = (C*)p; p += al(sizeof(C) * (size_t)B * k.M * k.N);
        C* v = (C*)p; p += al(sizeof(C) * (size_t)k.lam2 * k.L);
        C* wj = (C*)p; p += al(sizeof(C) * (size_t)k.lam2 * k.L);
        C* part = (C*)p;
        KTRY("zak_fwd", st, launch_zak_fwd<T>(f, f_real, k.L, zf, k.L, k.L, cg.d, *fd, nochirp(), B, st));
        KTRY("pre_ifft", st, launch_pre_ifft<T>((const C*)G, y, cg, k.lam2, *fft(cg.M), pp, B, st));
        KTRY("fft_grad_window", st, launch_fft_grad_window<T>(y, zf, k.lam2, v, part, cg, *fd, B, st));
        KTRY("zak_inv", st, launch_zak_inv<T>(v, k.L, wj, 0, k.L, k.L, cg.d, *fd, nochirp(), (T)1, k.lam2, st));
        KTRY("grad_window_combine", st, launch_grad_window_combine<T>(wj, grad, grad_real, k.L, k.a, k.lam2, (const int64_t*)sigma.p,
                                               cisL.tab, st));
        return DGT_OK;
    }

    // the power-of-two kernels read / write channels 0..M/2 directly: the FIR kernels, and
    // the channel FFT of the coset and time-shear routes (analysis) or its adjoint (synthesis)
    bool half_io(bool synthesis) const {
        const PlanCore& k = core;
        const bool p2row = k.M >= 128 && (k.M & (k.M - 1)) == 0 && k.M <= (int64_t)(sizeof(T) == 4 ? 16384 : 8192);
        if (k.route == DGT_ROUTE_FIR) return p2row && k.M <= 8192 && (!synthesis || k.fir_p2_synth);
        return p2row && !k.freq_shear && k.sep.M == k.M;
    }
    int exec_real(const void* f, void* ch, int64_t B, cudaStream_t st) override {
        if (!half_io(false)) return exec_real_via<T>(this, f, ch, B, st);
        DGT_TRY(real_ok(core));
        return exec_core(f, 1, ch, B, nullptr, st, true);
    }
    int iexec_real(const void* ch, void* f, int64_t B, int which, cudaStream_t st) override {
        if (!half_io(true)) return iexec_real_via<T>(this, ch, f, B, which, st);
        DGT_TRY(real_ok(core));
        return iexec_core(ch, f, 1, B, which, nullptr, expired, st, true);
    }

    // FIR synthesis whose seam scratch is the library's fixed per-GPU array: no allocation.
    int fir_synthesis_noalloc(const void* c, void* f, int f_real, int64_t B, int which, cudaStream_t st) override {
        const PlanCore& k = core;
        if (which < 0 || which > 2) return fail(DGT_ERR_ARG, "bad synthesis window %d", which);
        if (k.route != DGT_ROUTE_FIR) return fail(DGT_ERR_ARG, "allocation-free synthesis needs an FIR-route plan");
        if (!k.fir_synth_ok)
            return fail(DGT_ERR_UNSUPPORTED, "FIR synthesis: %lld columns per tile cannot cover a window of %lld",
                        (long long)k.fir_cols, (long long)k.Lg);
        if (!zg_ok[which])
            return fail(DGT_ERR_ARG, "the dual / tight window is not cached yet (call dgt_window_dual/_tight first)");
        if (B <= 0) return B == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
        FirParams<C> fp = fir_params(which);
        const size_t need = sizeof(C) * (size_t)B * fir_seam_elems(fp);
        if (need > kNoAllocScratchBytes)
            return fail(DGT_ERR_UNSUPPORTED, "allocation-free synthesis needs %zu bytes of scratch; the fixed array holds %zu",
                        need, kNoAllocScratchBytes);
        // the fixed array of the plan's device (its taps and tables live there too)
        int cur = -1;
        CUDA_TRY(cudaGetDevice(&cur));
        if (cur != k.device)
            return fail(DGT_ERR_ARG, "allocation-free synthesis on device %d for a plan of device %d: make the plan's "
                        "device current", cur, k.device);
        void* scratch = nullptr;
        CUDA_TRY(noalloc_scratch(&scratch));
        KTRY("fir_synthesis_noalloc", st, launch_fir_synthesis<T>((const C*)c, f, f_real, (C*)scratch, fp, *fft(k.M), B, st));
        return DGT_OK;
    }

    int logmag(const void* c, void* G, double* loss, double eps, int64_t B, cudaStream_t st) override {
        const PlanCore& k = core;
        DGT_TRY(lossparts.alloc(sizeof(double) * 64 * B));
        KTRY("logmag", st, launch_logmag<T>((const C*)c, (C*)G, (double*)lossparts.p, loss, k.M * k.N, (T)eps, B, st));
        return DGT_OK;
    }
};

// ---------------------------------------------------------------------------------------
// plan creation
// ---------------------------------------------------------------------------------------
static SepGeom make_sep(int64_t L, int64_t a, int64_t M) {
    SepGeom g{};
    g.L = L; g.a = a; g.M = M; g.b = L / M; g.N = L / a;
    g.c = igcd(a, M);
    g.d = igcd(g.b, g.N);
    g.p = a / g.c;
    g.q = M / g.c;
    g.K0 = L / g.d;
    return g;
}

static bool fft_ok(int64_t n, int precision) {
    FftPlanDev pl;
    if (!radix_plan(n, pl)) return false;
    return precision == DGT_F64 ? n + 1 <= tile_cap<double>() : n + 1 <= tile_cap<float>();
}
// lengths usable as the row length M of the Zak routes (fft_post / pre_ifft)
static bool fft_rows_ok(int64_t n, int precision) { return fft_ok(n, precision) || row_only_len_ok(n, precision); }

static int create_plan(dgt_plan_t* out, int64_t L, int64_t a, int64_t M, int64_t lam1, int64_t lam2, const dgt_window* g,
                       int route, int precision, cudaStream_t st, bool allow_fir = true) {
    if (!out || !g || !g->data) return fail(DGT_ERR_ARG, "null plan or window pointer");
    *out = nullptr;
    if (L <= 0 || a <= 0 || M <= 0 || lam2 <= 0) return fail(DGT_ERR_ARG, "L, a, M, lambda2 must be positive");
    if (lam1 < 0 || lam1 >= lam2 || igcd(lam1, lam2) != 1) return fail(DGT_ERR_ARG, "need 0 <= lambda1 < lambda2, gcd 1");
    if (L > ((int64_t)1 << 30)) return fail(DGT_ERR_UNSUPPORTED, "L above 2^30");
    if (L % a || L % M || L % (lam2 * ilcm(a, M)))
        return fail(DGT_ERR_LENGTH, "L=%lld is not a multiple of lambda2*lcm(a,M)=%lld", (long long)L,
                    (long long)(lam2 * ilcm(a, M)));
    if (precision != DGT_F32 && precision != DGT_F64) return fail(DGT_ERR_ARG, "bad precision");
    if (route < DGT_ROUTE_AUTO || route > DGT_ROUTE_FIR) return fail(DGT_ERR_ARG, "bad route");
    if (g->kind != DGT_WINDOW_FULL && g->kind != DGT_WINDOW_FIR) return fail(DGT_ERR_ARG, "bad window kind");
    if (g->kind == DGT_WINDOW_FULL && g->len != L) return fail(DGT_ERR_ARG, "full window needs len == L");
    if (g->kind == DGT_WINDOW_FIR && (g->len <= 0 || g->len > L / 2 || g->center < 0 || g->center >= g->len))
        return fail(DGT_ERR_ARG, "FIR window needs 0 < len <= L/2 and 0 <= center < len");

    PlanCore k{};
    k.L = L; k.a = a; k.M = M; k.lam1 = lam1; k.lam2 = lam2;
    k.b = L / M; k.N = L / a; k.s = k.b * lam1 / lam2;
    k.precision = precision;
    CUDA_TRY(cudaGetDevice(&k.device));
    k.win_kind = g->kind;
    k.Lg = g->len;
    k.center = g->kind == DGT_WINDOW_FIR ? g->center : 0;
    k.win_real = g->is_real;
    k.g_host.assign(2 * g->len, 0.0);
    for (int64_t i = 0; i < g->len; ++i) {
        k.g_host[2 * i] = g->is_real ? g->data[i] : g->data[2 * i];
        k.g_host[2 * i + 1] = g->is_real ? 0.0 : g->data[2 * i + 1];
    }
    k.coset_sep = make_sep(L, lam2 * a, M);

    // shear parameters (always computed; reported by dgt_plan_get_info)
    // a frequency shear with b_r = X runs the separable lattice (X, L / (a b / X)) of FFT(f)
    auto freq_sep_runs = [&](int64_t X) {
        const int64_t ar = a * k.b / X;
        const SepGeom sg = make_sep(L, X, L / ar);
        return fft_ok(sg.d, precision) && fft_rows_ok(sg.M, precision);
    };
    if (!shear_select(L, a, k.b, k.s, k.sh, freq_sep_runs)) return fail(DGT_ERR_ARG, "no shear found");
    k.freq_shear = k.sh.s0 != 0;

    // FIR chunking: columns per CTA, a divisor of N, fitting the shared-memory tile;
    // synthesis also needs a * cols >= Lg - a so that only neighbouring chunks overlap
    int64_t fir_cols = 0, fir_group = 1;
    bool fir_synth_ok = false;
    bool fir_p2 = false;
    if (g->kind == DGT_WINDOW_FIR && fft_ok(M, precision)) {
        const size_t csz = precision == DGT_F64 ? 16 : 8;
        const int64_t need = std::max<int64_t>(1, (g->len + a - 1) / a);
        // spare rows for the grouped FFT: the largest of 4, 2, 1 with which both the analysis
        // tile (rows + spare + input segment) and the synthesis tile (rows + spare) fit
        auto group_for = [&](int64_t cc) -> int64_t {
            for (int64_t grp : {4, 2, 1}) {
                if (grp > cc) continue;
                if (csz * ((size_t)(cc + grp) * (M + 1) + (size_t)(a * (cc - 1) + g->len)) <= kSmemBudget) return grp;
            }
            return 0;
        };
        for (int64_t cc = 64; cc >= 1 && !fir_cols; --cc)
            if (k.N % cc == 0 && cc >= need && group_for(cc)) fir_cols = cc;
        fir_synth_ok = fir_cols > 0;
        for (int64_t cc = 64; cc >= 1 && !fir_cols; --cc)
            if (k.N % cc == 0 && group_for(cc)) fir_cols = cc;
        if (fir_cols && !fir_synth_ok) fir_synth_ok = a * fir_cols >= g->len - a;
        fir_group = fir_cols ? group_for(fir_cols) : 1;
        // power-of-two M: the scatter-accumulate synthesis kernel takes wider chunks
        const int64_t cols2 = precision == DGT_F64 ? p2_fir_synthesis_cols<double>(M, k.N, a, g->len)
                                                   : p2_fir_synthesis_cols<float>(M, k.N, a, g->len);
        if (cols2 > 0) {
            fir_cols = cols2;
            fir_synth_ok = true;
            fir_group = 1;
            fir_p2 = true;
        }
    }
    if (route == DGT_ROUTE_AUTO) {
        if (allow_fir && g->kind == DGT_WINDOW_FIR && fir_cols && fir_synth_ok && lam2 <= 8) route = DGT_ROUTE_FIR;
        else route = k.freq_shear ? DGT_ROUTE_COSET : DGT_ROUTE_SHEAR;
    }
    if (route == DGT_ROUTE_FIR && g->kind != DGT_WINDOW_FIR)
        return fail(DGT_ERR_ARG, "the FIR route needs an FIR window");
    if (route != DGT_ROUTE_FIR && g->kind == DGT_WINDOW_FIR) {
        // full-window route with a short window: expand it
        std::vector<double> full(2 * L, 0.0);
        for (int64_t t = 0; t < g->len; ++t) {
            const int64_t l = pmod(t - g->center, L);
            full[2 * l] = k.g_host[2 * t];
            full[2 * l + 1] = k.g_host[2 * t + 1];
        }
        k.g_host.swap(full);
        k.win_kind = DGT_WINDOW_FULL;
        k.Lg = L;
        k.center = 0;
    }
    k.route = route;
    if (route != DGT_ROUTE_SHEAR) k.freq_shear = false;

    if (route == DGT_ROUTE_FIR) {
        if (!fft_ok(M, precision)) return fail(DGT_ERR_UNSUPPORTED, "FFT length M=%lld unsupported", (long long)M);
        if (lam2 > 8) return fail(DGT_ERR_UNSUPPORTED, "FIR route supports lambda2 <= 8");
        if (!fir_cols) return fail(DGT_ERR_UNSUPPORTED, "FIR route: M=%lld too long for one tile", (long long)M);
        k.fir_cols = fir_cols;
        k.fir_group = fir_group;
        k.fir_synth_ok = fir_synth_ok;
        k.fir_p2_synth = fir_p2;
    } else if (route == DGT_ROUTE_COSET) {
        k.sep = make_sep(L, lam2 * a, M);
        k.J = lam2;
    } else if (!k.freq_shear) {
        k.sep = make_sep(L, a, M);
        k.J = 1;
    } else {
        // frequency-side shear: separable DGT with time step b_r and N_r channels on FFT(f)
        const int64_t br = k.sh.b_r;
        k.ar = a * k.b / br;
        k.Mr = L / br;
        k.Nr = L / k.ar;
        k.C1 = k.ar / a;
        k.C2 = -(k.sh.s0 * br) / a;
        const int64_t twoN = 2 * k.N;
        k.C3m = (int64_t)((__int128)pmod(a * k.sh.s1, twoN) * ((L + 1) % twoN) % twoN);
        k.C4m = (int64_t)((__int128)pmod(k.C2 * br, twoN) * ((L + 1) % twoN) % twoN);
        k.C5m = pmod(2 * k.C1 * br, twoN);
        k.C6 = (int64_t)(((__int128)k.sh.s0 * k.sh.s1 + 1) * br % L);
        k.sep = make_sep(L, br, k.Nr);
        k.J = 1;
        // L = L1 L2, both transformable in one tile, as balanced as possible; a split into two
        // lengths with compiled mixed-radix transforms is preferred when there is one
        int64_t b1 = 0, bc = 0;
        for (int64_t x = 1; x * x <= L; ++x)
            if (L % x == 0 && fft_ok(x, precision) && fft_ok(L / x, precision)) {
                b1 = x;
                if (mr_compiled_len(x) && mr_compiled_len(L / x)) bc = x;
            }
        if (b1 == 0) return fail(DGT_ERR_UNSUPPORTED, "FFT_L split of L=%lld unsupported", (long long)L);
        if (bc) b1 = bc;
        k.L1 = b1;
        k.L2 = L / b1;
    }
    if (route != DGT_ROUTE_FIR) {
        if (!fft_ok(k.sep.d, precision) || !fft_rows_ok(k.sep.M, precision))
            return fail(DGT_ERR_UNSUPPORTED, "separable FFT lengths d=%lld, M=%lld unsupported", (long long)k.sep.d,
                        (long long)k.sep.M);
    }

    dgt_plan_s* p = nullptr;
    int s;
    if (precision == DGT_F32) {
        auto* q = new PlanImpl<float>();
        q->core = k;
        s = q->init(st);
        p = q;
    } else {
        auto* q = new PlanImpl<double>();
        q->core = k;
        s = q->init(st);
        p = q;
    }
    if (s == DGT_OK) s = expiry_word_take(&p->expired);
    if (s != DGT_OK) {
        delete p;
        return s;
    }
    *out = p;
    return DGT_OK;
}

// ---------------------------------------------------------------------------------------
// Blockwise (overlap-add) plan (Section 4, OLA; Section 4.1, shear-OLA): blocks of Lb samples,
// zero-extended to Lx, transformed by a full-window plan of length Lx, their coefficient
// columns added into the long transform's columns (and the adjoint for synthesis).
// ---------------------------------------------------------------------------------------
template <typename T> struct OlaPlan final : dgt_plan_s {
    using C = cplx<T>;
    std::unique_ptr<PlanImpl<T>> inner;
    OlaGeom og{};
    int64_t Lg = 0, center = 0;        // the FIR window (the blocks' plan holds it expanded to Lx)
    DevBuf work;

    struct Layout { size_t x, cx, in, total; };
    static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
    Layout layout(int64_t B) const {
        Layout ly{};
        ly.x = 0;
        ly.cx = al(sizeof(C) * (size_t)B * og.Nb * og.Lx);
        ly.in = ly.cx + al(sizeof(C) * (size_t)B * og.Nb * og.Nx * og.M);
        ly.total = ly.in + inner->ws_bytes(B * og.Nb);
        return ly;
    }
    char* workspace(int64_t B, void* wsp) {
        if (wsp) return (char*)wsp;
        if (work.alloc(layout(B).total) != DGT_OK) return nullptr;
        return (char*)work.p;
    }
    int exec(const void* f, int f_real, void* c, int64_t B, void* wsp, cudaStream_t st) override {
        if (B <= 0) return B == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
        const Layout ly = layout(B);
        char* ws = workspace(B, wsp);
        if (!ws) return DGT_ERR_OOM;
        KTRY("ola_split", st, launch_ola_split<T>(f, f_real, ws + ly.x, og, B, st));
        DGT_TRY(inner->exec(ws + ly.x, f_real, ws + ly.cx, B * og.Nb, ws + ly.in, st));
        KTRY("ola_add", st, launch_ola_add<T>((const C*)(ws + ly.cx), (C*)c, og, B, st));
        return DGT_OK;
    }
    int iexec(const void* c, void* f, int f_real, int64_t B, int which, void* wsp, unsigned int* expired,
              cudaStream_t st) override {
        if (which < 0 || which > 2) return fail(DGT_ERR_ARG, "bad synthesis window %d", which);
        if (B <= 0) return B == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
        if (which) {
            if (wsp && !inner->zg_ok[which])
                return fail(DGT_ERR_ARG, "the dual / tight window is not cached yet (call dgt_window_dual/_tight)");
            DGT_TRY(inner->ensure_window(which, st));
        }
        const Layout ly = layout(B);
        char* ws = workspace(B, wsp);
        if (!ws) return DGT_ERR_OOM;
        KTRY("ola_gather", st, launch_ola_gather<T>((const C*)c, (C*)(ws + ly.cx), og, B, st));
        DGT_TRY(inner->iexec(ws + ly.cx, ws + ly.x, f_real, B * og.Nb, which, ws + ly.in, expired, st));
        KTRY("ola_take", st, launch_ola_take<T>(ws + ly.x, f_real, f, og, B, st));
        return DGT_OK;
    }
    // the window on Z_L: the local window's taps moved from Z_Lx to Z_L (the dual of a window
    // no longer than M is the same on both: S is diagonal with the same a-periodic weights)
    int window_out(int which, void* out, cudaStream_t st) override {
        const PlanCore& k = core;
        DevBuf loc;
        DGT_TRY(loc.alloc(sizeof(C) * (size_t)og.Lx));
        DGT_TRY(inner->window_out(which, loc.p, st));
        std::vector<T> lw(2 * og.Lx), gw(2 * k.L, (T)0);
        CUDA_TRY(cudaMemcpyAsync(lw.data(), loc.p, sizeof(C) * og.Lx, cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int64_t t = 0; t < Lg; ++t) {
            const int64_t li = pmod(t - center, og.Lx), gi = pmod(t - center, k.L);
            gw[2 * gi] = lw[2 * li];
            gw[2 * gi + 1] = lw[2 * li + 1];
        }
        CUDA_TRY(cudaMemcpyAsync(out, gw.data(), sizeof(C) * k.L, cudaMemcpyHostToDevice, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return DGT_OK;
    }
    int set_window(const void*, int, cudaStream_t) override {
        return fail(DGT_ERR_UNSUPPORTED, "blockwise plans keep the window they were created with");
    }
    int grad_window(const void*, int, const void*, void*, int, int64_t, cudaStream_t) override {
        return fail(DGT_ERR_UNSUPPORTED, "window gradient needs a full-length window");
    }
    int logmag(const void*, void*, double*, double, int64_t, cudaStream_t) override {
        return fail(DGT_ERR_UNSUPPORTED, "use a plain plan of the same lattice for the loss helper");
    }
    int fir_synthesis_noalloc(const void*, void*, int, int64_t, int, cudaStream_t) override {
        return fail(DGT_ERR_ARG, "allocation-free synthesis needs an FIR-route plan");
    }
    int exec_real(const void* f, void* ch, int64_t B, cudaStream_t st) override {
        return exec_real_via<T>(this, f, ch, B, st);
    }
    int iexec_real(const void* ch, void* f, int64_t B, int which, cudaStream_t st) override {
        return iexec_real_via<T>(this, ch, f, B, which, st);
    }
    size_t ws_bytes(int64_t B) const override { return layout(B).total; }
    size_t owned_bytes() const override { return inner->owned_bytes() + work.bytes + real_full.bytes; }
};

static int create_ola_plan(dgt_plan_t* out, int64_t L, int64_t a, int64_t M, int64_t lam1, int64_t lam2,
                           const dgt_window* g, int64_t Lb, int inner_route, int precision, cudaStream_t st) {
    if (!out || !g || !g->data) return fail(DGT_ERR_ARG, "null plan or window pointer");
    *out = nullptr;
    if (g->kind != DGT_WINDOW_FIR) return fail(DGT_ERR_ARG, "blockwise plans need an FIR window");
    if (inner_route != DGT_ROUTE_AUTO && inner_route != DGT_ROUTE_COSET && inner_route != DGT_ROUTE_SHEAR)
        return fail(DGT_ERR_ARG, "blockwise plans run the coset or the shear route on the blocks");
    if (L <= 0 || a <= 0 || M <= 0 || lam2 <= 0 || Lb <= 0) return fail(DGT_ERR_ARG, "sizes must be positive");
    if (lam1 < 0 || lam1 >= lam2 || igcd(lam1, lam2) != 1) return fail(DGT_ERR_ARG, "need 0 <= lambda1 < lambda2, gcd 1");
    const int64_t q = lam2 * ilcm(a, M);
    if (L % q) return fail(DGT_ERR_LENGTH, "L=%lld is not a multiple of lambda2*lcm(a,M)=%lld", (long long)L, (long long)q);
    if (L % Lb || Lb % q)
        return fail(DGT_ERR_LENGTH, "block length %lld must divide L and be a multiple of lambda2*lcm(a,M)=%lld",
                    (long long)Lb, (long long)q);
    if (g->len <= 0 || g->center < 0 || g->center >= g->len) return fail(DGT_ERR_ARG, "bad FIR window");
    if (Lb < g->len) return fail(DGT_ERR_ARG, "the block must be at least as long as the window");
    // the smallest admissible length Lx >= Lb + Lg whose transform this build supports (FFT
    // lengths with prime factors up to 7, tiles that fit)
    int64_t Lx = (Lb + g->len + q - 1) / q * q;
    if (Lx > L) return fail(DGT_ERR_LENGTH, "the extended block (%lld) is longer than the signal", (long long)Lx);
    dgt_plan_t in = nullptr;
    for (int tries = 0;; ++tries, Lx += q) {
        if (Lx > L || tries == 64)
            return fail(DGT_ERR_UNSUPPORTED, "no supported block transform length from %lld", (long long)(Lb + g->len));
        const int s = create_plan(&in, Lx, a, M, lam1, lam2, g, inner_route, precision, st, /*allow_fir=*/false);
        if (s == DGT_OK) break;
        if (s != DGT_ERR_UNSUPPORTED) return s;
    }
    OlaGeom og{};
    og.L = L; og.a = a; og.M = M; og.N = L / a; og.Lb = Lb; og.Nb = L / Lb; og.Lx = Lx; og.Nx = Lx / a;
    og.S = Lb / a; og.nu_hi = (Lb - 1 + g->center) / a;
    og.K = std::min<int64_t>(og.Nb, (og.Nx + og.S - 1) / og.S + 1);
    PlanCore k = in->core;
    k.L = L; k.N = L / a; k.b = L / M; k.s = k.b * lam1 / lam2;
    k.ola_block = Lb;
    k.ola_len = Lx;
    if (precision == DGT_F32) {
        auto* p = new OlaPlan<float>();
        p->inner.reset(static_cast<PlanImpl<float>*>(in));
        p->og = og;
        p->Lg = g->len;
        p->center = g->center;
        p->core = k;
        *out = p;
    } else {
        auto* p = new OlaPlan<double>();
        p->inner.reset(static_cast<PlanImpl<double>*>(in));
        p->og = og;
        p->Lg = g->len;
        p->center = g->center;
        p->core = k;
        *out = p;
    }
    if (const int e = expiry_word_take(&(*out)->expired)) {
        delete *out;
        *out = nullptr;
        return e;
    }
    return DGT_OK;
}

// ---------------------------------------------------------------------------------------
// Two-dimensional DGT on a tensor-product lattice (Section 3.5): the plan of the second axis
// on every row, a transpose, the plan of the first axis on every column of the result, a
// transpose; synthesis in the reverse order.
// ---------------------------------------------------------------------------------------
struct dgt2_plan_s {
    std::unique_ptr<dgt_plan_s> p1, p2;   // first axis (L1), second axis (L2)
    int64_t L1 = 0, L2 = 0, K1 = 0, K2 = 0;   // K = N M coefficients per axis
    int precision = DGT_F32;
    DevBuf work;
    static size_t al(size_t x) { return (x + 255) & ~(size_t)255; }

    template <typename T> int exec(const void* f, int f_real, void* c, int64_t B, cudaStream_t st) {
        using C = cplx<T>;
        const size_t n12 = (size_t)B * L1 * K2, n3 = (size_t)B * K1 * K2;
        DGT_TRY(work.alloc(2 * al(sizeof(C) * n12) + al(sizeof(C) * n3)));
        C* t1 = (C*)work.p;
        C* t2 = (C*)((char*)work.p + al(sizeof(C) * n12));
        C* t3 = (C*)((char*)work.p + 2 * al(sizeof(C) * n12));
        DGT_TRY(p2->exec(f, f_real, t1, B * L1, nullptr, st));                 // rows: [B][L1][N2 M2]
        KTRY("transpose", st, launch_transpose<T>(t1, t2, L1, K2, B, st));      // [B][N2 M2][L1]
        DGT_TRY(p1->exec(t2, 0, t3, B * K2, nullptr, st));                      // [B][N2 M2][N1 M1]
        KTRY("transpose", st, launch_transpose<T>(t3, (C*)c, K2, K1, B, st));   // [B][N1 M1][N2 M2]
        return DGT_OK;
    }
    template <typename T> int iexec(const void* c, void* f, int f_real, int64_t B, int which, cudaStream_t st) {
        using C = cplx<T>;
        const size_t n12 = (size_t)B * L1 * K2, n3 = (size_t)B * K1 * K2;
        DGT_TRY(work.alloc(2 * al(sizeof(C) * n12) + al(sizeof(C) * n3)));
        C* t1 = (C*)work.p;
        C* t2 = (C*)((char*)work.p + al(sizeof(C) * n12));
        C* t3 = (C*)((char*)work.p + 2 * al(sizeof(C) * n12));
        KTRY("transpose", st, launch_transpose<T>((const C*)c, t3, K1, K2, B, st));   // [B][N2 M2][N1 M1]
        DGT_TRY(p1->iexec(t3, t2, 0, B * K2, which, nullptr, p1->expired, st));     // [B][N2 M2][L1]
        KTRY("transpose", st, launch_transpose<T>(t2, t1, K2, L1, B, st));           // [B][L1][N2 M2]
        return p2->iexec(t1, f, f_real, B * L1, which, nullptr, p2->expired, st);   // [B][L1][L2]
    }
};

// ---------------------------------------------------------------------------------------
// host-buffer pipeline: the batch in chunks of `chunk` signals through two device staging
// slots.  Chunk i is copied in on the pipe's input stream, transformed on the caller's stream
// and copied out on the pipe's output stream, so the copies of chunks i + 1 and i - 1 overlap
// the transform of chunk i.  A slot is refilled only after the transform of the chunk two
// earlier has read it, and rewritten only after that chunk's copy out.  The whole call is
// ordered after the caller's earlier work on `st`, and the caller's later work waits for the
// last copy out.
// ---------------------------------------------------------------------------------------
static int host_pipeline(dgt_plan_t plan, const void* in_h, size_t bin, void* out_h, size_t bout, int64_t batch,
                         int64_t chunk, cudaStream_t st,
                         const std::function<int(const void*, void*, int64_t)>& run) {
    if (batch <= 0) return batch == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
    if (chunk < 0) return fail(DGT_ERR_ARG, "negative chunk");
    int dev = -1;
    CUDA_TRY(cudaGetDevice(&dev));
    if (plan->core.device >= 0 && dev != plan->core.device)
        return fail(DGT_ERR_ARG, "the current device (%d) is not the plan's (%d)", dev, plan->core.device);
    DGT_TRY(plan->pending_expiry());
    if (!plan->host_pipe) plan->host_pipe.reset(new HostPipe());
    HostPipe& hp = *plan->host_pipe;
    DGT_TRY(hp.init());
    const int64_t ch = chunk > 0 && chunk < batch ? chunk : batch;
    const int64_t nchunks = (batch + ch - 1) / ch;
    const int slots = nchunks > 1 ? 2 : 1;
    for (int s = 0; s < slots; ++s) {
        DGT_TRY(hp.src[s].alloc(bin * (size_t)ch));
        DGT_TRY(hp.dst[s].alloc(bout * (size_t)ch));
    }
    CUDA_TRY(cudaEventRecord(hp.start, st));
    CUDA_TRY(cudaStreamWaitEvent(hp.in, hp.start, 0));
    CUDA_TRY(cudaStreamWaitEvent(hp.out, hp.start, 0));
    for (int64_t i = 0; i < nchunks; ++i) {
        const int s = (int)(i & 1);
        const int64_t nb = std::min(ch, batch - i * ch);
        if (i >= 2) CUDA_TRY(cudaStreamWaitEvent(hp.in, hp.done_exec[s], 0));
        CUDA_TRY(cudaMemcpyAsync(hp.src[s].p, (const char*)in_h + (size_t)(i * ch) * bin, (size_t)nb * bin,
                                 cudaMemcpyHostToDevice, hp.in));
        CUDA_TRY(cudaEventRecord(hp.done_in[s], hp.in));
        CUDA_TRY(cudaStreamWaitEvent(st, hp.done_in[s], 0));
        if (i >= 2) CUDA_TRY(cudaStreamWaitEvent(st, hp.done_out[s], 0));
        DGT_TRY(run(hp.src[s].p, hp.dst[s].p, nb));
        CUDA_TRY(cudaEventRecord(hp.done_exec[s], st));
        CUDA_TRY(cudaStreamWaitEvent(hp.out, hp.done_exec[s], 0));
        CUDA_TRY(cudaMemcpyAsync((char*)out_h + (size_t)(i * ch) * bout, hp.dst[s].p, (size_t)nb * bout,
                                 cudaMemcpyDeviceToHost, hp.out));
        CUDA_TRY(cudaEventRecord(hp.done_out[s], hp.out));
    }
    CUDA_TRY(cudaEventRecord(hp.last, hp.out));
    CUDA_TRY(cudaStreamWaitEvent(st, hp.last, 0));
    return DGT_OK;
}

// ---------------------------------------------------------------------------------------
// extern "C"
// ---------------------------------------------------------------------------------------
extern "C" {

int dgt_plan_create(dgt_plan_t* plan, int64_t L, int64_t a, int64_t M, int64_t lambda1, int64_t lambda2,
                    const dgt_window* g, int route, int precision, void* stream) {
    try {
        return create_plan(plan, L, a, M, lambda1, lambda2, g, route, precision, (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fail(DGT_ERR_OOM, "host allocation failed");
    }
}

int dgt_plan_create_ola(dgt_plan_t* plan, int64_t L, int64_t a, int64_t M, int64_t lambda1, int64_t lambda2,
                        const dgt_window* g, int64_t block_len, int inner_route, int precision, void* stream) {
    try {
        return create_ola_plan(plan, L, a, M, lambda1, lambda2, g, block_len, inner_route, precision,
                               (cudaStream_t)stream);
    } catch (const std::bad_alloc&) {
        return fail(DGT_ERR_OOM, "host allocation failed");
    }
}

int dgt2_plan_create(dgt2_plan_t* plan, int64_t L1, int64_t a1, int64_t M1, int64_t lam11, int64_t lam12,
                     const dgt_window* g1, int64_t L2, int64_t a2, int64_t M2, int64_t lam21, int64_t lam22,
                     const dgt_window* g2, int route, int precision, void* stream) {
    if (!plan) return fail(DGT_ERR_ARG, "null plan pointer");
    *plan = nullptr;
    try {
        dgt_plan_t q1 = nullptr, q2 = nullptr;
        DGT_TRY(create_plan(&q1, L1, a1, M1, lam11, lam12, g1, route, precision, (cudaStream_t)stream));
        std::unique_ptr<dgt_plan_s> h1(q1);
        DGT_TRY(create_plan(&q2, L2, a2, M2, lam21, lam22, g2, route, precision, (cudaStream_t)stream));
        auto* p = new dgt2_plan_s();
        p->p1 = std::move(h1);
        p->p2.reset(q2);
        p->L1 = L1; p->L2 = L2;
        p->K1 = (L1 / a1) * M1; p->K2 = (L2 / a2) * M2;
        p->precision = precision;
        *plan = p;
        return DGT_OK;
    } catch (const std::bad_alloc&) {
        return fail(DGT_ERR_OOM, "host allocation failed");
    }
}

int dgt2_exec(dgt2_plan_t plan, const void* f, int f_is_real, void* c, int64_t batch, void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    if (batch <= 0) return batch == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
    return plan->precision == DGT_F64 ? plan->exec<double>(f, f_is_real, c, batch, (cudaStream_t)stream)
                                      : plan->exec<float>(f, f_is_real, c, batch, (cudaStream_t)stream);
}

int idgt2_exec(dgt2_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window, void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    if (which_window < 0 || which_window > 2) return fail(DGT_ERR_ARG, "bad synthesis window %d", which_window);
    if (batch <= 0) return batch == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
    return plan->precision == DGT_F64 ? plan->iexec<double>(c, f, f_real_out, batch, which_window, (cudaStream_t)stream)
                                      : plan->iexec<float>(c, f, f_real_out, batch, which_window, (cudaStream_t)stream);
}

int dgt2_plan_status(dgt2_plan_t plan, void* stream) {
    if (!plan) return fail(DGT_ERR_ARG, "null plan");
    DGT_TRY(plan->p1->status_check((cudaStream_t)stream));
    return plan->p2->status_check((cudaStream_t)stream);
}

void dgt2_plan_destroy(dgt2_plan_t plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    delete plan;
}

int dgt_plan_get_info(dgt_plan_t plan, dgt_plan_info* info) {
    if (!plan || !info) return fail(DGT_ERR_ARG, "null pointer");
    const PlanCore& k = plan->core;
    memset(info, 0, sizeof(*info));
    info->L = k.L; info->a = k.a; info->M = k.M; info->lambda1 = k.lam1; info->lambda2 = k.lam2;
    info->b = k.b; info->N = k.N; info->s = k.s;
    info->route = k.route;
    info->precision = k.precision;
    info->s0 = k.sh.s0; info->s1 = k.sh.s1; info->b_r = k.sh.b_r;
    info->sep_a = k.sep.a; info->sep_M = k.sep.M;
    info->c = k.sep.c; info->d = k.sep.d; info->p = k.sep.p; info->q = k.sep.q;
    info->n_windows = k.J;
    info->fir_len = k.route == DGT_ROUTE_FIR ? k.Lg : 0;
    info->ola_block = k.ola_block;
    info->ola_len = k.ola_len;
    return DGT_OK;
}

int dgt_plan_set_window(dgt_plan_t plan, const void* g_dev, int is_real, void* stream) {
    if (!plan || !g_dev) return fail(DGT_ERR_ARG, "null pointer");
    return plan->set_window(g_dev, is_real, (cudaStream_t)stream);
}

int dgt_exec(dgt_plan_t plan, const void* f, int f_is_real, void* c, int64_t batch, void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    DGT_TRY(plan->pending_expiry());
    return plan->exec(f, f_is_real, c, batch, nullptr, (cudaStream_t)stream);
}

int idgt_exec(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window, void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    DGT_TRY(plan->pending_expiry());
    return plan->iexec(c, f, f_real_out, batch, which_window, nullptr, plan->expired, (cudaStream_t)stream);
}

int idgt_exec_window(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, const void* gamma,
                     int gamma_is_real, void* stream) {
    if (!plan || !gamma || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    DGT_TRY(plan->pending_expiry());
    return plan->iexec_window(c, f, f_real_out, batch, gamma, gamma_is_real, (cudaStream_t)stream);
}

int dgt_exec_real(dgt_plan_t plan, const void* f, void* c, int64_t batch, void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    DGT_TRY(plan->pending_expiry());
    return plan->exec_real(f, c, batch, (cudaStream_t)stream);
}

int idgt_exec_real(dgt_plan_t plan, const void* c, void* f, int64_t batch, int which_window, void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    if (which_window < 0 || which_window > 2) return fail(DGT_ERR_ARG, "bad synthesis window %d", which_window);
    DGT_TRY(plan->pending_expiry());
    return plan->iexec_real(c, f, batch, which_window, (cudaStream_t)stream);
}

int dgt_workspace_bytes(dgt_plan_t plan, int64_t batch, size_t* bytes) {
    if (!plan || !bytes || batch < 0) return fail(DGT_ERR_ARG, "bad argument");
    *bytes = kWsHeader + plan->ws_bytes(batch);
    return DGT_OK;
}

int dgt_exec_host(dgt_plan_t plan, const void* f, int f_is_real, void* c, int64_t batch, int64_t chunk, void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    const PlanCore& k = plan->core;
    const size_t rs = k.precision == DGT_F64 ? sizeof(double) : sizeof(float);
    const size_t bin = (f_is_real ? rs : 2 * rs) * (size_t)k.L, bout = 2 * rs * (size_t)k.N * (size_t)k.M;
    cudaStream_t st = (cudaStream_t)stream;
    return host_pipeline(plan, f, bin, c, bout, batch, chunk, st, [&](const void* din, void* dout, int64_t nb) {
        return plan->exec(din, f_is_real, dout, nb, nullptr, st);
    });
}

int idgt_exec_host(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window,
                   int64_t chunk, void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    const PlanCore& k = plan->core;
    const size_t rs = k.precision == DGT_F64 ? sizeof(double) : sizeof(float);
    const size_t bin = 2 * rs * (size_t)k.N * (size_t)k.M, bout = (f_real_out ? rs : 2 * rs) * (size_t)k.L;
    cudaStream_t st = (cudaStream_t)stream;
    return host_pipeline(plan, c, bin, f, bout, batch, chunk, st, [&](const void* din, void* dout, int64_t nb) {
        return plan->iexec(din, dout, f_real_out, nb, which_window, nullptr, plan->expired, st);
    });
}

int dgt_exec_ws(dgt_plan_t plan, const void* f, int f_is_real, void* c, int64_t batch, void* workspace, void* stream) {
    if (!plan || (!f && batch) || (!c && batch) || !workspace) return fail(DGT_ERR_ARG, "null pointer");
    if (((uintptr_t)workspace) & 255) return fail(DGT_ERR_ARG, "workspace must be 256-byte aligned");
    return plan->exec(f, f_is_real, c, batch, (char*)workspace + kWsHeader, (cudaStream_t)stream);
}

int idgt_exec_ws(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window,
                 void* workspace, void* stream) {
    if (!plan || (!f && batch) || (!c && batch) || !workspace) return fail(DGT_ERR_ARG, "null pointer");
    if (((uintptr_t)workspace) & 255) return fail(DGT_ERR_ARG, "workspace must be 256-byte aligned");
    if (batch <= 0) return batch == 0 ? DGT_OK : fail(DGT_ERR_ARG, "negative batch");
    // this call's expiry word: the first word of the workspace, cleared in stream order
    CUDA_TRY(cudaMemsetAsync(workspace, 0, sizeof(unsigned int), (cudaStream_t)stream));
    return plan->iexec(c, f, f_real_out, batch, which_window, (char*)workspace + kWsHeader, (unsigned int*)workspace,
                       (cudaStream_t)stream);
}

int dgt_workspace_status(dgt_plan_t plan, const void* workspace, void* stream) {
    if (!plan || !workspace) return fail(DGT_ERR_ARG, "null pointer");
    unsigned int w = 0;
    CUDA_TRY(cudaMemcpyAsync(&w, workspace, sizeof(w), cudaMemcpyDeviceToHost, (cudaStream_t)stream));
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    CUDA_TRY(cudaGetLastError());
    if (w) {
        CUDA_TRY(cudaMemsetAsync(const_cast<void*>(workspace), 0, sizeof(w), (cudaStream_t)stream));
        return fail(DGT_ERR_TIMEOUT, "a synthesis kernel of this workspace's call gave up waiting for its tile copies");
    }
    return DGT_OK;
}

int dgt_window_dual(dgt_plan_t plan, void* gamma_out, void* stream) {
    if (!plan || !gamma_out) return fail(DGT_ERR_ARG, "null pointer");
    return plan->window_out(1, gamma_out, (cudaStream_t)stream);
}

int dgt_window_tight(dgt_plan_t plan, void* gt_out, void* stream) {
    if (!plan || !gt_out) return fail(DGT_ERR_ARG, "null pointer");
    return plan->window_out(2, gt_out, (cudaStream_t)stream);
}

int dgt_grad_window(dgt_plan_t plan, const void* f, int f_is_real, const void* G, void* grad_g, int grad_real,
                    int64_t batch, void* stream) {
    if (!plan || !f || !G || !grad_g || batch <= 0) return fail(DGT_ERR_ARG, "bad argument");
    DGT_TRY(plan->pending_expiry());
    return plan->grad_window(f, f_is_real, G, grad_g, grad_real, batch, (cudaStream_t)stream);
}

int dgt_fir_synthesis_noalloc(dgt_plan_t plan, const void* c, void* f, int f_real_out, int64_t batch, int which_window,
                              void* stream) {
    if (!plan || (!f && batch) || (!c && batch)) return fail(DGT_ERR_ARG, "null pointer");
    DGT_TRY(plan->pending_expiry());
    return plan->fir_synthesis_noalloc(c, f, f_real_out, batch, which_window, (cudaStream_t)stream);
}

int dgt_logmag_loss(dgt_plan_t plan, const void* c, void* G, double* loss_dev, double eps, int64_t batch, void* stream) {
    if (!plan || !c || !loss_dev || batch <= 0) return fail(DGT_ERR_ARG, "bad argument");
    DGT_TRY(plan->pending_expiry());
    return plan->logmag(c, G, loss_dev, eps, batch, (cudaStream_t)stream);
}

int dgt_plan_bytes(dgt_plan_t plan, size_t* bytes) {
    if (!plan || !bytes) return fail(DGT_ERR_ARG, "null pointer");
    *bytes = plan->owned_bytes();
    return DGT_OK;
}

int dgt_plan_status(dgt_plan_t plan, void* stream) {
    if (!plan) return fail(DGT_ERR_ARG, "null plan");
    return plan->status_check((cudaStream_t)stream);
}

int dgt_debug_touch_guard(dgt_plan_t plan) {
    if (!plan) return fail(DGT_ERR_ARG, "null plan");
    const int r = plan->debug_touch_guard();
    if (r == DGT_ERR_UNSUPPORTED) return fail(r, "guard zones exist only in the DGT_DEBUG build");
    return r == DGT_OK ? DGT_OK : fail(r, "could not write the guard zone");
}

int dgt_sync(void* stream) {
    CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
    CUDA_TRY(cudaGetLastError());
    int n = 0;
    {
        std::lock_guard<std::mutex> lock(g_expiry_mu);
        for (unsigned int* w : g_expiry_live) n += expiry_word_take_value(w) ? 1 : 0;
    }
    if (n) return fail(DGT_ERR_TIMEOUT, "synthesis kernels of %d plans gave up waiting for their tile copies", n);
    return DGT_OK;
}

long long dgt_chirp_table_cap(long long bytes) {
    const long long old = g_chirp_cap;
    if (bytes >= 0) g_chirp_cap = bytes;
    return old;
}

long long dgt_wait_limit(long long cycles) {
    const long long old = g_wait_limit_cycles;
    if (cycles >= 0) g_wait_limit_cycles = cycles;
    return old;
}

void dgt_plan_destroy(dgt_plan_t plan) {
    if (!plan) return;
    cudaDeviceSynchronize();
    delete plan;
}

const char* dgt_strerror(int status) {
    switch (status) {
        case DGT_OK: return "DGT_OK";
        case DGT_ERR_ARG: return "DGT_ERR_ARG";
        case DGT_ERR_LENGTH: return "DGT_ERR_LENGTH";
        case DGT_ERR_NOT_FRAME: return "DGT_ERR_NOT_FRAME";
        case DGT_ERR_CUDA: return "DGT_ERR_CUDA";
        case DGT_ERR_OOM: return "DGT_ERR_OOM";
        case DGT_ERR_TIMEOUT: return "DGT_ERR_TIMEOUT";
        case DGT_ERR_UNSUPPORTED: return "DGT_ERR_UNSUPPORTED";
        default: return "DGT_ERR_UNKNOWN";
    }
}

const char* dgt_last_error(void) { return g_last_error.c_str(); }

int dgt_profile_start(void) {
    g_prof.clear();
    g_prof_used = 0;
    g_prof_on = true;
    return DGT_OK;
}

int dgt_profile_stop(char* json, size_t cap) {
    g_prof_on = false;
    CUDA_TRY(cudaDeviceSynchronize());
    std::map<std::string, std::pair<int64_t, double>> acc;
    for (const ProfRec& r : g_prof) {
        float ms = 0;
        CUDA_TRY(cudaEventElapsedTime(&ms, r.a, r.b));
        auto& v = acc[r.name];
        v.first += 1;
        v.second += ms;
    }
    std::string out = "{";
    bool first = true;
    for (auto& kv : acc) {
        char buf[256];
        snprintf(buf, sizeof(buf), "%s\"%s\": {\"launches\": %lld, \"ms\": %.6f}", first ? "" : ", ",
                 kv.first.c_str(), (long long)kv.second.first, kv.second.second);
        out += buf;
        first = false;
    }
    out += "}";
    g_prof.clear();
    g_prof_used = 0;
    if (json && cap) {
        strncpy(json, out.c_str(), cap - 1);
        json[cap - 1] = 0;
        if (out.size() >= cap) return fail(DGT_ERR_ARG, "profile buffer too small (%zu bytes needed)", out.size() + 1);
    }
    return DGT_OK;
}

int dgt_fma_rate(int kind, double* flops_per_s, void* stream) {
    if (!flops_per_s || kind < 0 || kind > 2) return fail(DGT_ERR_ARG, "bad argument");
    int dev = 0, sms = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    DevBuf sink;
    DGT_TRY(sink.alloc(sizeof(float)));
    // 8 resident CTAs of 256 threads per SM; about 10 ms of float work
    const int iters = kind == 2 ? 1 << 12 : 1 << 16;
    CUDA_TRY(fma_rate(kind, iters, 8 * sms, (float*)sink.p, (cudaStream_t)stream, flops_per_s));
    return DGT_OK;
}

int dgt_fft_selftest(int64_t n, int precision, int direction, const void* in, void* out, int64_t howmany, void* stream) {
    if (!in || !out || howmany < 0 || (direction != -1 && direction != 1)) return fail(DGT_ERR_ARG, "bad argument");
    cudaStream_t st = (cudaStream_t)stream;
    if (precision == DGT_F32) {
        TwTable<float> t;
        if (!radix_plan(n, t.ref.pl) || n + 1 > tile_cap<float>())
            return fail(DGT_ERR_UNSUPPORTED, "length %lld", (long long)n);
        DGT_TRY(upload_cplx<float>(t.buf, twiddle_host(n), st));
        t.ref.tw = t.buf.p;
        KTRY("fft_rows_test", st, launch_fft_rows_test<float>((const float2*)in, (float2*)out, t.ref, direction, howmany, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    } else {
        TwTable<double> t;
        if (!radix_plan(n, t.ref.pl) || n + 1 > tile_cap<double>())
            return fail(DGT_ERR_UNSUPPORTED, "length %lld", (long long)n);
        DGT_TRY(upload_cplx<double>(t.buf, twiddle_host(n), st));
        t.ref.tw = t.buf.p;
        KTRY("fft_rows_test", st, launch_fft_rows_test<double>((const double2*)in, (double2*)out, t.ref, direction, howmany, st));
        CUDA_TRY(cudaStreamSynchronize(st));
    }
    return DGT_OK;
}

}  // extern "C"
