// cr_device.cuh -- device-side helpers shared by the cyclic-reduction kernels.
//
// Complex numbers are double2 (x = real, y = imaginary), the byte layout of
// crsolve_z / complex128.  Every complex multiply-add is written as four
// fused multiply-adds: on GB300 the FP64 pipe (2 DFMA per clock per SM) is the
// bound of the whole FP64 path, so the kernels count FP64 instructions, not
// bytes.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace crs {

typedef double2 z2;
typedef float2 c2;

// complex type of a real type
template <class R> struct Cplx;
template <> struct Cplx<double> { using type = double2; };
template <> struct Cplx<float> { using type = float2; };
template <class R> using cplx_t = typename Cplx<R>::type;

#define CRS_NO_FAIL 0xFFFFFFFFFFFFFFFFull

__device__ __forceinline__ double fmx(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fmx(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double rsq(double v) { return rsqrt(v); }
__device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }
__device__ __forceinline__ double qnan(double) { return __longlong_as_double(0x7ff8000000000000ll); }
__device__ __forceinline__ float qnan(float) { return __int_as_float(0x7fc00000); }

__device__ __forceinline__ z2 zmk(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ c2 zmk(float re, float im) { return make_float2(re, im); }
template <class C> __device__ __forceinline__ C zsub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <class C, class R> __device__ __forceinline__ C zscale(C a, R s) { C r; r.x = a.x * s; r.y = a.y * s; return r; }
// Negation by flipping the sign bit on the integer pipe.  The XOR is written
// in PTX so that the compiler cannot turn it back into a floating-point
// negation, which it would issue as a DADD on the FP64 pipe, the pipe that
// bounds the FP64 kernels.  Exact, so results are unchanged.
__device__ __forceinline__ double dneg_bits(double v) {
    int hi = __double2hiint(v);
    const int lo = __double2loint(v);
    asm("xor.b32 %0, %0, 0x80000000;" : "+r"(hi));
    return __hiloint2double(hi, lo);
}
__device__ __forceinline__ float dneg_bits(float v) { return __int_as_float(__float_as_int(v) ^ (int)0x80000000u); }
// Sign flipped when sgn = 0x80000000, unchanged when sgn = 0 (a runtime
// choice without a branch or a floating-point instruction).
__device__ __forceinline__ double flip_if(double v, unsigned sgn) {
    int hi = __double2hiint(v);
    const int lo = __double2loint(v);
    asm("xor.b32 %0, %0, %1;" : "+r"(hi) : "r"(sgn));
    return __hiloint2double(hi, lo);
}
__device__ __forceinline__ float flip_if(float v, unsigned sgn) { return __int_as_float(__float_as_int(v) ^ (int)sgn); }
template <class C> __device__ __forceinline__ C zneg(C a) { C r; r.x = dneg_bits(a.x); r.y = dneg_bits(a.y); return r; }
template <class C> __device__ __forceinline__ C zconj(C a) { C r = a; r.y = dneg_bits(a.y); return r; }

// acc -= a * b
template <class C> __device__ __forceinline__ void zmsub(C &acc, C a, C b) {
    acc.x = fmx(-a.x, b.x, acc.x);
    acc.x = fmx(a.y, b.y, acc.x);
    acc.y = fmx(-a.x, b.y, acc.y);
    acc.y = fmx(-a.y, b.x, acc.y);
}
// acc -= a * conj(b)
template <class C> __device__ __forceinline__ void zmsub_cb(C &acc, C a, C b) {
    acc.x = fmx(-a.x, b.x, acc.x);
    acc.x = fmx(-a.y, b.y, acc.x);
    acc.y = fmx(-a.y, b.x, acc.y);
    acc.y = fmx(a.x, b.y, acc.y);
}
// acc -= conj(a) * b
template <class C> __device__ __forceinline__ void zmsub_ca(C &acc, C a, C b) {
    acc.x = fmx(-a.x, b.x, acc.x);
    acc.x = fmx(-a.y, b.y, acc.x);
    acc.y = fmx(-a.x, b.y, acc.y);
    acc.y = fmx(a.y, b.x, acc.y);
}
// acc += a * b
template <class C> __device__ __forceinline__ void zmac(C &acc, C a, C b) {
    acc.x = fmx(a.x, b.x, acc.x);
    acc.x = fmx(-a.y, b.y, acc.x);
    acc.y = fmx(a.x, b.y, acc.y);
    acc.y = fmx(a.y, b.x, acc.y);
}
// acc += a * conj(b)
template <class C> __device__ __forceinline__ void zmac_cb(C &acc, C a, C b) {
    acc.x = fmx(a.x, b.x, acc.x);
    acc.x = fmx(a.y, b.y, acc.x);
    acc.y = fmx(a.y, b.x, acc.y);
    acc.y = fmx(-a.x, b.y, acc.y);
}
// acc += conj(a) * b
template <class C> __device__ __forceinline__ void zmac_ca(C &acc, C a, C b) {
    acc.x = fmx(a.x, b.x, acc.x);
    acc.x = fmx(a.y, b.y, acc.x);
    acc.y = fmx(a.x, b.y, acc.y);
    acc.y = fmx(-a.y, b.x, acc.y);
}

// Record a breakdown: the smallest (level, 1-based local block) key wins.
__device__ __forceinline__ void report_fail(unsigned long long *status, int level, int64_t local1) {
    atomicMin(status, ((unsigned long long)level << 40) | (unsigned long long)local1);
}

// Row p of the lower triangle that holds flat index f = p(p+1)/2 + q, q <= p.
__device__ __forceinline__ int tri_row(int f) {
    int p = (int)((sqrtf(8.0f * (float)f + 1.0f) - 1.0f) * 0.5f);
    while ((p + 1) * (p + 2) / 2 <= f) ++p;
    while (p * (p + 1) / 2 > f) --p;
    return p;
}

// Arguments of one reduction level (Sec. 2 eq. Formulas on a level with Nl
// blocks; odd blocks t = 0..no-1 sit at 0-based position 2t, even blocks
// j' = 0..ne-1 at 2j'+1), in real type R (double: the FP64 path; float: the
// FP32 levels of the mixed-precision path).
template <class R>
struct LevelArgsT {
    using C = cplx_t<R>;
    int64_t Nl, no, ne;
    int m, k, nb, kc, level;
    int inline_fix;     // 1: one CTA runs the chunks of the level in order and completes each
                        // chunk-boundary even block itself (no Wbd / cbd, no fix-up pass)
    unsigned *bd_count; // nullable: one arrival counter per chunk boundary (per right-hand-side
                        // chunk in the down sweep), zero on entry; the second CTA to arrive at a
                        // boundary completes its even block (see bd_arrive), no fix-up pass
    const C *A;         // [Nl][m][m] level system (lower triangle read)
    const C *B;         // [Nl-1][m][m]
    C *L;               // [no][m][m]  Cholesky factors (lower, upper zero)
    R *inv;             // [no][m]     1 / diag(L)
    C *Z;               // [no][m][2m] [P | Q] = L^{-1} [B_{i-1} | B_i^H]
    C *Wbd;             // [ncta][m][m] P^H P of each CTA's first odd block (CTA-boundary scratch)
    C *An;              // [ne][m][m]  next level diagonal blocks
    C *Bn;              // [ne-1][m][m] next level sub-diagonal blocks
    const C *y;         // [Nl][m][k]  level right-hand side
    C *r;               // [no][m][k]  L^{-1} y_odd
    C *cbd;             // [ncta][m][k] P^H r of each CTA's first odd block (CTA-boundary scratch)
    C *yn;              // [ne][m][k]  next level right-hand side
    const C *xn;        // [ne][m][k]  next level solution
    C *x;               // [Nl][m][k]  level solution
    unsigned long long *status;
    int *err;           // nullable: set to 1 if a bounded device-side wait gave up
    // Breakdown index map (see report_index): 0 for classic reduction; for the
    // concatenated split systems of Algorithm 1, rep_bits = log2 N and rep_off
    // the position of this reduction's block 0 in the level's concatenation.
    int64_t rep_off;
    int rep_bits;
    // Chunk range of one launch of the odd-block kernels: chunks c_begin ..
    // c_begin + c_count - 1 (c_count = 0: every chunk of the level).  A level
    // may be run as several such launches, e.g. each as soon as the input
    // rows it reads are complete.  For the factor fix-up kernel the same
    // fields give the range of chunk boundaries (c_count = 0: 1 .. chunks-1).
    int64_t c_begin, c_count;
    // Bounds-checked builds (CRSOLVE_DEBUG_BOUNDS): the first out-of-range
    // access is recorded here (see dbg_in); nullptr otherwise.
    unsigned long long *dbg;
};
using LevelArgs = LevelArgsT<double>;

// Arrays of a level, for the bounds checks of debug builds.
enum DbgArray { kDbgA = 1, kDbgB, kDbgL, kDbgInv, kDbgZ, kDbgWbd, kDbgAn, kDbgBn, kDbgY, kDbgR, kDbgCbd, kDbgYn,
                kDbgXn, kDbgX, kDbgResid };


// Element count of array `which` of a level, from the level sizes alone:
// A [Nl][m][m], B [Nl-1][m][m], L [no][m][m], inv [no][m], Z [no][m][2m],
// Wbd [ctas][m][m], An [ne][m][m], Bn [ne-1][m][m], y and x [Nl][m][k],
// r [no][m][k], cbd [ctas][m][k], yn and xn [ne][m][k].
template <class R>
__device__ __forceinline__ int64_t dbg_extent(const LevelArgsT<R> &a, int which) {
    const int64_t mm = (int64_t)a.m * a.m, mk = (int64_t)a.m * a.k;
    const int64_t ctas = a.nb > 0 ? (a.no + a.nb - 1) / a.nb : 0;
    switch (which) {
        case kDbgA: return a.Nl * mm;
        case kDbgB: return (a.Nl > 1 ? a.Nl - 1 : 0) * mm;
        case kDbgL: return a.no * mm;
        case kDbgInv: return a.no * a.m;
        case kDbgZ: return a.no * 2 * mm;
        case kDbgWbd: return ctas * mm;
        case kDbgAn: return a.ne * mm;
        case kDbgBn: return (a.ne > 1 ? a.ne - 1 : 0) * mm;
        case kDbgY: case kDbgX: return a.Nl * mk;
        case kDbgR: return a.no * mk;
        case kDbgCbd: return ctas * mk;
        case kDbgYn: case kDbgXn: return a.ne * mk;
        default: return 0;
    }
}

// Debug builds: is idx inside array `which`?  If not, the first such access
// (smallest record: level, array, index) is kept in *a.dbg and the caller
// skips the access (a load gives zero), so a faulty index never touches
// memory.  Release builds: always true, no code.
#ifdef CRSOLVE_DEBUG_BOUNDS
template <class R>
__device__ __forceinline__ bool dbg_in(const LevelArgsT<R> &a, int which, int64_t idx) {
    if (idx >= 0 && idx < dbg_extent(a, which)) return true;
    if (a.dbg) {
        const unsigned long long rec = ((unsigned long long)(a.level & 0xFF) << 56) |
                                       ((unsigned long long)which << 48) |
                                       ((unsigned long long)idx & 0xFFFFFFFFFFFFull);
        atomicMin(a.dbg, rec);
    }
    return false;
}
#define CRS_IN(a, which, idx) (::crs::dbg_in((a), ::crs::which, (int64_t)(idx)))
#else
#define CRS_IN(a, which, idx) (true)
#endif

// 1-based block index that a breakdown of the level block at 0-based position
// pos0 reports.  Classic reduction: the local index pos0 + 1.  Algorithm 1
// (rep_bits = L = log2 N): level l holds the 2^l split systems of size N/2^l
// one after another, each split putting the odd half before the even half, so
// position p of the concatenation holds original block rotl^l(p) (rotation on
// L bits); that original index is reported.
template <class R>
__device__ __forceinline__ int64_t report_index(const LevelArgsT<R> &a, int64_t pos0) {
    if (a.rep_bits == 0) return pos0 + 1;
    const int nb = a.rep_bits, s = a.level % nb;
    const uint64_t mask = (1ull << nb) - 1;
    const uint64_t u = (uint64_t)(pos0 + a.rep_off) & mask;
    const uint64_t r = s ? (((u << s) | (u >> (nb - s))) & mask) : u;
    return (int64_t)r + 1;
}

}  // namespace crs
