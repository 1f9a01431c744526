// Complex arithmetic on float2 / double2 and exact phase tables.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace dgt {

template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };
template <typename T> using cplx = typename CT<T>::type;

template <typename C> struct RealOf;
template <> struct RealOf<float2> { using type = float; };
template <> struct RealOf<double2> { using type = double; };

__host__ __device__ __forceinline__ float2 mk(float x, float y) { return make_float2(x, y); }
__host__ __device__ __forceinline__ double2 mk(double x, double y) { return make_double2(x, y); }

template <typename C> __host__ __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __host__ __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 1000 && !defined(DGT_SCALAR_F32)
#define DGT_PACKED_F32 1
// float: one packed two-lane instruction per complex addition (same rounding per lane as the
// scalar forms; a - b is the fused b * (-1) + a, which is exact before its one rounding).
// -DDGT_SCALAR_F32 builds the scalar forms instead.
template <> __device__ __forceinline__ float2 cadd<float2>(float2 a, float2 b) { return __fadd2_rn(a, b); }
template <> __device__ __forceinline__ float2 csub<float2>(float2 a, float2 b) {
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}
// a + s i b for s = +-1: (a.x - s b.y, a.y + s b.x), one packed fused multiply-add
template <int S> __device__ __forceinline__ float2 cadd_ib(float2 a, float2 b) {
    return __ffma2_rn(make_float2(b.y, b.x), make_float2((float)-S, (float)S), a);
}
#endif
template <typename C> __host__ __device__ __forceinline__ C cmul(C a, C b) {
    C r;
    r.x = a.x * b.x - a.y * b.y;
    r.y = a.x * b.y + a.y * b.x;
    return r;
}
// a * conj(b)
template <typename C> __host__ __device__ __forceinline__ C cmulc(C a, C b) {
    C r;
    r.x = a.x * b.x + a.y * b.y;
    r.y = a.y * b.x - a.x * b.y;
    return r;
}
template <typename C> __host__ __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename R> __host__ __device__ __forceinline__ C cscale(C a, R s) {
#ifdef DGT_PACKED_F32
    if constexpr (sizeof(C) == 8) return __fmul2_rn(a, make_float2((float)s, (float)s));
#endif
    a.x *= s;
    a.y *= s;
    return a;
}
// multiply by +i (DIR=+1) or -i (DIR=-1)
template <int DIR, typename C> __host__ __device__ __forceinline__ C mul_i(C a) {
    C r;
    if (DIR > 0) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
    return r;
}

// x mod d for 64-bit x and a fixed divisor 1 <= d < 2^32 without a hardware division:
// Barrett reduction with m = floor((2^64 - 1) / d); the quotient estimate umulhi(x, m)
// is at most 2 below floor(x / d), so two conditional subtractions finish it.
struct ModU64 {
    uint64_t d;
    uint64_t m;
    __host__ __device__ __forceinline__ uint64_t mod(uint64_t x) const {
#ifdef __CUDA_ARCH__
        const uint64_t q = __umul64hi(x, m);
#else
        const uint64_t q = (uint64_t)(((unsigned __int128)x * m) >> 64);
#endif
        uint64_t r = x - q * d;
        if (r >= d) r -= d;
        if (r >= d) r -= d;
        return r;
    }
    // signed argument, result in [0, d)
    __host__ __device__ __forceinline__ uint64_t smod(int64_t x) const {
        if (x >= 0) return mod((uint64_t)x);
        const uint64_t r = mod((uint64_t)(-x));
        return r ? d - r : 0;
    }
    // (x * y) mod d for 0 <= x, y < d
    __host__ __device__ __forceinline__ uint64_t mulmod(uint64_t x, uint64_t y) const { return mod(x * y); }
    // floor(x / d), same estimate and corrections
    __host__ __device__ __forceinline__ uint64_t div(uint64_t x) const {
#ifdef __CUDA_ARCH__
        uint64_t q = __umul64hi(x, m);
#else
        uint64_t q = (uint64_t)(((unsigned __int128)x * m) >> 64);
#endif
        uint64_t r = x - q * d;
        if (r >= d) { ++q; r -= d; }
        if (r >= d) ++q;
        return q;
    }
};

inline ModU64 make_mod(uint64_t d) {
    ModU64 r;
    r.d = d;
    r.m = ~(uint64_t)0 / d;
    return r;
}

// 32-bit form for arguments below 2^32: quotient estimate floor(x m / 2^32) with
// m = floor((2^32 - 1) / d), which is short by at most two (two corrections)
struct ModU32 {
    uint32_t d;
    uint32_t m;
    __device__ __forceinline__ uint32_t div(uint32_t x) const {
        uint32_t q = __umulhi(x, m);
        uint32_t r = x - q * d;
        if (r >= d) { r -= d; ++q; }
        if (r >= d) ++q;
        return q;
    }
    __device__ __forceinline__ uint32_t mod(uint32_t x) const {
        const uint32_t q = __umulhi(x, m);
        uint32_t r = x - q * d;
        if (r >= d) r -= d;
        if (r >= d) r -= d;
        return r;
    }
};
inline ModU32 make_mod32(uint32_t d) {
    ModU32 r;
    r.d = d;
    r.m = 0xffffffffu / d;
    return r;
}

// exp(2 pi i e / den) for integer e (any sign), from a two-level table built on the
// host in double precision: hi[k] = exp(2 pi i k S / den), lo[r] = exp(2 pi i r / den),
// e mod den = k S + r with S a power of two.  Two rounded factors, so the result is
// accurate to a few ulp of the working precision, independent of the size of den.
template <typename C> struct CisTable {
    const C* hi;
    const C* lo;
    ModU64 md;            // modulus den
    int shift;            // S = 2^shift
    __device__ __forceinline__ C operator()(int64_t e) const {
        const uint64_t r = md.smod(e);
        return cmul(__ldg(hi + (r >> shift)), __ldg(lo + (r & ((1ull << shift) - 1))));
    }
    __device__ __forceinline__ C at(uint64_t r) const {      // 0 <= r < den
        return cmul(__ldg(hi + (r >> shift)), __ldg(lo + (r & ((1ull << shift) - 1))));
    }
};

// (x * y) mod m for 0 <= x, y < m <= 2^32
__host__ __device__ __forceinline__ uint64_t mulmod(uint64_t x, uint64_t y, uint64_t m) { return (x * y) % m; }
__host__ __device__ __forceinline__ int64_t posmod(int64_t x, int64_t m) {
    int64_t r = x % m;
    return r < 0 ? r + m : r;
}

}  // namespace dgt
