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

#define CRS_NO_FAIL 0xFFFFFFFFFFFFFFFFull

__device__ __forceinline__ z2 zmk(double re, double im) { return make_double2(re, im); }
__device__ __forceinline__ z2 zconj(z2 a) { return make_double2(a.x, -a.y); }
// negation by flipping sign bits (integer pipe, no FP64 instruction)
__device__ __forceinline__ double dneg_bits(double v) {
    return __longlong_as_double(__double_as_longlong(v) ^ (long long)0x8000000000000000ull);
}
__device__ __forceinline__ z2 zneg(z2 a) { return make_double2(dneg_bits(a.x), dneg_bits(a.y)); }
__device__ __forceinline__ z2 zscale(z2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ __forceinline__ z2 zsub(z2 a, z2 b) { return make_double2(a.x - b.x, a.y - b.y); }

// acc -= a * b
__device__ __forceinline__ void zmsub(z2 &acc, z2 a, z2 b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
}
// acc -= a * conj(b)
__device__ __forceinline__ void zmsub_cb(z2 &acc, z2 a, z2 b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(-a.y, b.x, acc.y);
    acc.y = fma(a.x, b.y, acc.y);
}
// acc -= conj(a) * b
__device__ __forceinline__ void zmsub_ca(z2 &acc, z2 a, z2 b) {
    acc.x = fma(-a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(-a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__device__ __forceinline__ void zmac_ca(z2 &acc, z2 a, z2 b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(-a.y, b.x, acc.y);
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
// j' = 0..ne-1 at 2j'+1).
struct LevelArgs {
    int64_t Nl, no, ne;
    int m, k, nb, kc, level;
    int inline_fix;     // 1: one CTA runs the chunks of the level in order and completes each
                        // chunk-boundary even block itself (no Wbd / cbd, no fix-up pass)
    const z2 *A;        // [Nl][m][m] level system (lower triangle read)
    const z2 *B;        // [Nl-1][m][m]
    z2 *L;              // [no][m][m]  Cholesky factors (lower, upper zero)
    double *inv;        // [no][m]     1 / diag(L)
    z2 *Z;              // [no][m][2m] [P | Q] = L^{-1} [B_{i-1} | B_i^H]
    z2 *Wbd;            // [ncta][m][m] P^H P of each CTA's first odd block (CTA-boundary scratch)
    z2 *An;             // [ne][m][m]  next level diagonal blocks
    z2 *Bn;             // [ne-1][m][m] next level sub-diagonal blocks
    const z2 *y;        // [Nl][m][k]  level right-hand side
    z2 *r;              // [no][m][k]  L^{-1} y_odd
    z2 *cbd;            // [ncta][m][k] P^H r of each CTA's first odd block (CTA-boundary scratch)
    z2 *yn;             // [ne][m][k]  next level right-hand side
    const z2 *xn;       // [ne][m][k]  next level solution
    z2 *x;              // [Nl][m][k]  level solution
    unsigned long long *status;
};

}  // namespace crs
