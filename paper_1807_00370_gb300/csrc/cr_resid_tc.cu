// cr_resid_tc.cu -- the FP64 residual r = y - A x of the block-tridiagonal
// system of eq. Axb on the BF16 tensor cores, by exact splitting (the
// error-free transformation of Ozaki, Ogita, Oishi and Rump, "Error-free
// transformations of matrix multiplication by using fast routines of matrix
// multiplication and its applications", Numer. Algorithms 59, 2012).
//
// The iterative refinement of the mixed-precision form needs residuals to
// FP64 accuracy; on GB300 the FP64 pipe runs at 1/64 of the FP32 rate, so the
// plain FP64 residual costs about a quarter of a whole FP64 solve at m = 64.
// Here every product is formed exactly on the tensor cores instead:
//
//   * Complex to real: block row j of A x is one real product
//       [Re r; Im r] = [[Re M, -Im M], [Im M, Re M]] [Re x; Im x]
//     with M the concatenation [B_{j-1} | A_j | B_j^H] (A_j Hermitian from its
//     lower triangle) and x the stack [x_{j-1}; x_j; x_{j+1}]: M = 128 rows
//     (real parts of the m <= 64 output rows, then imaginary parts), K = 3 *
//     2 * 64 = 384 (each complex column s contributes K indices 2s (times
//     Re x) and 2s+1 (times Im x)), N = 32 right-hand-side columns per pass.
//   * Exact splitting: every row of the real matrix gets one exponent E (the
//     largest binary exponent in the row), every column of the x stack one
//     exponent F.  A matrix entry v becomes the 60-bit integer
//     Q = round(|v| / 2^(E-59)), cut into ten 6-bit slices q_0..q_9 (most
//     significant first); an x entry the 54-bit integer round(|x| / 2^(F-53))
//     in nine slices t_0..t_8.  Each slice, with the entry's sign, is an
//     integer |q| <= 63, exact in BF16.  Entries within 2^-7 of their row's
//     largest are represented exactly (all 53 bits); smaller ones to half a
//     unit of 2^-60 of it.  The matrix grid is finer than the x grid on
//     purpose: a representation error of the matrix is the same in every
//     refinement step, so the refinement converges to the solution of the
//     perturbed matrix and the error is multiplied by kappa; an error of x
//     changes with x and is not.
//   * Products: for every slice pair (i, j) with d = i + j <= 11 the MMA
//     accumulates q_i t_j into the FP32 accumulator acc_d in tensor memory
//     (69 of the 90 pairs).  A diagonal holds at most 9 pairs, so |acc_d| <=
//     9 * 384 * 63^2 < 2^24: every partial sum is an exact integer in FP32
//     and the accumulators hold the exact sums.  Slice i is multiplied by the
//     x slices t_0..t_{min(8, 11-i)} in one MMA (two when that is wider than
//     256 columns) whose accumulator address is acc_i, so each product lands
//     in acc_{i+j}.  The dropped pairs i + j >= 12 are below 2^-62 of the
//     product of any entry within 2^-7 of its row's largest and its x.  (With
//     d <= 9 they were ~2^-53 of such products, and always of the same sign as
//     the product: a systematic shrink of A that refinement converges to and
//     kappa amplifies, 8.6e-11 at kappa ~ 1e6.)
//   * Epilogue (integer): A x = T 2^(E + F - 76) with the exact integer
//     T = sum_d acc_d 2^(6(11-d)) (128-bit); y goes onto the same grid and
//     r = y - A x is formed exactly in 128-bit integers and rounded once.
//     So the residual is more precise than an FP64 one (whose products and
//     sums each round): besides the final rounding only the rounding of
//     entries onto their grids and the dropped pairs remain.  Iterative
//     refinement with such a residual is not limited to kappa * u_FP64
//     (Carson and Higham's extra-precise residual).
//
// Data flow per CTA (persistent over block rows, one CTA per SM).  With the
// matrix slices precomputed once per factorisation (an image in the
// shared-memory layout, CRSOLVE_RESIDUAL_SPLIT_IMAGE, the mixed form's
// method): k_residual_ws, warp-specialised, streams the images through a
// four-stage ring (see there).  Without: k_residual_tc, where 16 warps cut a
// K-chunk of 32 into slices in shared memory (double-buffered, K-major, no
// swizzle) while one thread issues the MMAs of the previous chunk
// (tcgen05.mma kind::f16, BF16 inputs, FP32 accumulation in tensor memory)
// and commits them to the chunk buffer's mbarrier; after the last chunk all
// warps read the twelve accumulators back (tcgen05.ld) and write r.  Every
// mbarrier wait is bounded; on a timeout the kernel records the error, waits
// (bounded) for its MMAs and copies, frees tensor memory and returns.
#include "crsolve.h"
#include "cr_launch.h"
#include "cr_tc.cuh"

namespace crs {
namespace {

constexpr int kRtM = 128;                                // MMA rows
constexpr int kRtNSA = 10;                               // slices of a matrix entry (60-bit grid)
constexpr int kRtNSX = 9;                                // slices of an x entry (54-bit grid)
constexpr int kRtND = 12;                                // slice-product diagonals d = i + j kept
constexpr int kRtNC = 32;                                // right-hand-side columns per pass
constexpr int kRtKC = 32;                                // real K per chunk (16 complex columns)
constexpr int kRtASlice = kRtM * kRtKC * 2;              // 8192 bytes per matrix slice per chunk
constexpr int kRtAStage = kRtNSA * kRtASlice;            // 81920 bytes of matrix slices per chunk
constexpr int kRtBStage = kRtNSX * kRtNC * kRtKC * 2;    // 18432 bytes of x slices per chunk
constexpr int kRtStage = kRtAStage + kRtBStage;
constexpr int kRtThreads = 512;
constexpr int kRtTmemCols = 512;                         // twelve accumulators of 32 columns (384), rounded
constexpr int kExpZero = -4096, kExpNonFinite = 4096;    // exponent of an all-zero / non-finite set
constexpr int kRtWaitPolls = 1 << 24;

// Binary exponent e of v (|v| < 2^(e+1)), kExpZero for 0, kExpNonFinite for
// Inf / NaN.
__device__ __forceinline__ int dexp(double v) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int eb = (int)((b >> 52) & 0x7FF);
    if (eb == 0x7FF) return kExpNonFinite;
    if ((b & 0x7FFFFFFFFFFFFFFFull) == 0) return kExpZero;
    return eb == 0 ? -1022 : eb - 1023;
}

// |v| on the grid 2^(E + 1 - G) of a row or column with exponent E (G bits,
// |v| < 2^(E+1)), rounded to the nearest grid point: exact for entries within
// 2^(53-G) of the largest, and half a grid unit at most below that.  Values
// that round (they are below 2^(E+1-G+53)) cannot reach 2^G.
template <int G>
__device__ __forceinline__ unsigned long long fixq(double v, int E) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const int eb = (int)((b >> 52) & 0x7FF);
    unsigned long long S = b & 0x000FFFFFFFFFFFFFull;
    int e = -1022;
    if (eb != 0) {
        S |= 1ull << 52;
        e = eb - 1023;
    }
    const int sh = e - E + G - 53;    // <= G - 53 since e <= E
    if (sh >= 0) return S << sh;
    if (sh < -54) return 0;
    return (S + (1ull << (-sh - 1))) >> (-sh);
}

// FP32 bits of the signed integer (mag 0..63, sign from base): base is
// 0x4B000000 (2^23) with the entry's sign bit, off = -2^23 with the same
// sign, so (2^23 + mag) - 2^23 = mag exactly; its high 16 bits are the BF16
// value (exact: 6 significant bits).  Integer and FP32 pipes only.
__device__ __forceinline__ uint32_t f32_int(uint32_t mag, uint32_t base, float off) {
    return __float_as_uint(__uint_as_float(base | mag) + off);
}
// The high halves of two FP32 words as a BF16 pair (lo in the low half).
__device__ __forceinline__ uint32_t bf16_pair(uint32_t lo, uint32_t hi) { return __byte_perm(lo, hi, 0x7632); }
// Sign bit of a double from its bits (no FP64 instruction).
__device__ __forceinline__ uint32_t dsign(double v) { return (uint32_t)((unsigned long long)__double_as_longlong(v) >> 63) << 31; }

// Byte offset of element (r, k) of a K-major, unswizzled tile of 16-bit
// elements with kRtKC columns: core matrices of 8 rows x 8 elements (16 bytes
// per row, 128 bytes per core matrix), K-adjacent cores 128 bytes apart,
// 8-row groups (kRtKC / 8) * 128 = 512 bytes apart.
__device__ __forceinline__ int kmaj16(int r, int k) {
    return (r >> 3) * 512 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// Chunk entry e of the matrix part (64 rows i x 16 complex columns sl) and of
// the x part (16 rows sl x 32 columns c).  A warp's 32 consecutive e cover 8
// rows (or columns) mod 8 x 4 K-pairs mod 4, so its 32 shared-memory words
// fall in 32 different banks; its loads are 64-byte row pieces or 128-byte
// column pieces.
__device__ __forceinline__ int a_row(int e) { return ((e >> 7) << 3) | ((e >> 2) & 7); }
__device__ __forceinline__ int a_col(int e) { return (((e >> 5) & 3) << 2) | (e & 3); }
__device__ __forceinline__ int x_col(int e) { return (((e >> 5) & 3) << 3) | ((e >> 2) & 7); }
__device__ __forceinline__ int x_row(int e) { return ((e >> 7) << 2) | (e & 3); }

__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    // kind::f16 instruction descriptor: FP32 accumulator (bits 4-5 = 1), A and
    // B BF16 (bits 7-9, 10-12 = 1), both K-major, N >> 3 at bit 17, M >> 4 at 24
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(tmem_d),
        "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

// 16 consecutive columns of the calling warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
                 : "r"(taddr));
}

// 4 consecutive columns of the calling warp's 32 TMEM lanes.
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
                 : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;"); }

// One arrival on the mbarrier that also announces `bytes` of transaction count.
__device__ __forceinline__ void mbar_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Bulk copy of `bytes` (a multiple of 16, both addresses 16-byte aligned) from
// global to this CTA's shared memory, completing on the mbarrier.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}

// 2^e as a double (0 below the subnormal range, Inf above the normal one).
__device__ __forceinline__ double pow2(int e) {
    if (e >= -1022 && e <= 1023) return __longlong_as_double((long long)(e + 1023) << 52);
    return ldexp(1.0, e);
}

// Bounds-checked builds: is idx inside A [N][m][m] (which = kDbgA), B
// [N-1][m][m] (kDbgB) or a block vector [N][m][k] (kDbgResid)?  The first
// out-of-range access is recorded in *a.dbg (level field 0xFF) and skipped.
__device__ __forceinline__ bool rin(const ResidTcArgs &a, int which, int64_t idx) {
#ifdef CRSOLVE_DEBUG_BOUNDS
    const int64_t mm = (int64_t)a.m * a.m;
    const int64_t ext = which == kDbgA ? a.N * mm : which == kDbgB ? (a.N > 1 ? a.N - 1 : 0) * mm
                                                                   : a.N * (int64_t)a.m * a.k;
    if (idx >= 0 && idx < ext) return true;
    if (a.dbg)
        atomicMin(a.dbg, (0xFFull << 56) | ((unsigned long long)which << 48) | ((unsigned long long)idx & 0xFFFFFFFFFFFFull));
    return false;
#else
    (void)a;
    (void)which;
    (void)idx;
    return true;
#endif
}

// The product's fixed-point sum T (an exact integer) and y,
// combined into r = y - T 2^se with a single rounding: y goes onto the same
// grid 2^se (exactly, unless its bits reach below the grid, which lies about
// 2^-66 of the product's largest term under it), the difference is formed
// exactly as a 128-bit integer and rounded to the nearest double (ties to
// even).  Returns false (and the caller falls back to FP64 arithmetic) for a
// non-finite y, a y far above the product, or a result outside the normal
// double range.
__device__ __forceinline__ bool resid_exact(double y, __int128 T, int se, double &out) {
    const unsigned long long yb = (unsigned long long)__double_as_longlong(y);
    const int eyb = (int)((yb >> 52) & 0x7FF);
    if (eyb == 0x7FF) return false;
    unsigned long long My = yb & 0x000FFFFFFFFFFFFFull;
    int ey = -1022;
    if (eyb != 0) {
        My |= 1ull << 52;
        ey = eyb - 1023;
    }
    const int sy = ey - 52 - se;     // y = My 2^sy on the grid 2^se
    __int128 Y = 0;
    if (My != 0) {
        if (sy > 60) return false;
        if (sy >= 0) Y = (__int128)My << sy;
        else if (sy > -60) Y = (__int128)((My + (1ull << (-sy - 1))) >> (-sy));
    }
    if (yb >> 63) Y = -Y;
    const __int128 R = Y - T;
    if (R == 0) {
        out = 0.0;
        return true;
    }
    const bool neg = R < 0;
    const unsigned __int128 U = neg ? (unsigned __int128)(-R) : (unsigned __int128)R;
    const unsigned long long hi = (unsigned long long)(U >> 64), lo = (unsigned long long)U;
    const int nbits = hi ? 128 - __clzll((long long)hi) : 64 - __clzll((long long)lo);
    int sh = nbits - 53;
    unsigned long long mant;
    if (sh <= 0) {
        mant = lo << (-sh);
    } else {
        mant = (unsigned long long)(U >> sh);
        const unsigned __int128 rem = U - ((unsigned __int128)mant << sh);
        const unsigned __int128 half = (unsigned __int128)1 << (sh - 1);
        if (rem > half || (rem == half && (mant & 1ull))) ++mant;
        if (mant == (1ull << 53)) {
            mant >>= 1;
            ++sh;
        }
    }
    const int e = 52 + sh + se;      // the value is mant 2^(sh + se), mant in [2^52, 2^53)
    if (e < -1022 || e > 1023) return false;
    out = __longlong_as_double((long long)(((unsigned long long)neg << 63) |
                                           ((unsigned long long)(e + 1023) << 52) | (mant & 0x000FFFFFFFFFFFFFull)));
    return true;
}

// Entry (i, s) of the complex block b of row j's coupling row
// [B_{j-1} | A_j | B_j^H]: zero outside the matrix.
__device__ __forceinline__ z2 coupling(const ResidTcArgs &a, int64_t j, int b, int i, int s) {
    const int m = a.m;
    const int64_t mm = (int64_t)m * m;
    if (i >= m || s >= m) return zmk(0.0, 0.0);
    if (b == 0) {
        const int64_t o = (j - 1) * mm + (int64_t)i * m + s;
        if (j == 0 || !rin(a, kDbgB, o)) return zmk(0.0, 0.0);
        return __ldg(a.B + o);
    }
    if (b == 1) {
        const int64_t o = j * mm + (s <= i ? (int64_t)i * m + s : (int64_t)s * m + i);
        if (!rin(a, kDbgA, o)) return zmk(0.0, 0.0);
        if (s < i) return __ldg(a.A + o);
        if (s == i) return zmk(__ldg(&a.A[o].x), 0.0);
        return zconj(__ldg(a.A + o));        // sign flip on the integer pipe
    }
    const int64_t o = j * mm + (int64_t)s * m + i;
    if (j + 1 >= a.N || !rin(a, kDbgB, o)) return zmk(0.0, 0.0);
    return zconj(__ldg(a.B + o));
}

// Cut matrix entry v (row i, complex column sl of a K-chunk; row exponent E)
// into its ten slices and store them as BF16 pairs in the ten tiles at dst
// (shared memory, or a precomputed image in global memory with the same
// layout): real row i gets (Re M, -Im M), imaginary row i + 64 (Im M, Re M).
__device__ __forceinline__ void slice_matrix_entry(z2 v, int E, int i, int sl, unsigned char *dst) {
    const unsigned long long qr = fixq<60>(v.x, E), qi = fixq<60>(v.y, E);
    const uint32_t sr = dsign(v.x), si = dsign(v.y);
    const uint32_t baser = 0x4B000000u | sr, basei = 0x4B000000u | si;
    const float offr = __uint_as_float(0xCB000000u ^ sr), offi = __uint_as_float(0xCB000000u ^ si);
    const int o_re = kmaj16(i, 2 * sl), o_im = kmaj16(i + 64, 2 * sl);
#pragma unroll
    for (int n = 0; n < kRtNSA; ++n) {
        const int sh = 54 - 6 * n;
        const uint32_t mr = (uint32_t)(qr >> sh) & 63u, mi = (uint32_t)(qi >> sh) & 63u;
        const uint32_t fr = f32_int(mr, baser, offr), fi = f32_int(mi, basei, offi);
        unsigned char *An = dst + n * kRtASlice;
        *reinterpret_cast<uint32_t *>(An + o_re) = bf16_pair(fr, fi ^ 0x80000000u);
        *reinterpret_cast<uint32_t *>(An + o_im) = bf16_pair(fi, fr);
    }
}

__global__ void __launch_bounds__(256) k_row_exponents(ResidTcArgs a) {
    const int m = a.m;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.N * m; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / m;
        const int i = (int)(e - j * m);
        int E = kExpZero;
        for (int b = 0; b < 3; ++b)
            for (int s = 0; s < m; ++s) {
                const z2 v = coupling(a, j, b, i, s);
                E = max(E, max(dexp(v.x), dexp(v.y)));
            }
        a.erow[e] = E;
    }
}

__global__ void __launch_bounds__(256) k_col_exponents(ResidTcArgs a) {
    const int m = a.m, k = a.k;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < a.N * k; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / k;
        const int c = (int)(e - j * k);
        int F = kExpZero;
        for (int i = 0; i < m; ++i) {
            const z2 v = __ldg(a.x + (j * m + i) * (int64_t)k + c);
            F = max(F, max(dexp(v.x), dexp(v.y)));
        }
        a.ecol[e] = F;
    }
}

// ------------------------------------------------ image path, warp-specialised
//
// With the matrix slices precomputed (an image per block row and K-chunk of
// 16, in the shared-memory layout), the residual is a stream of bulk copies
// into tensor-core products.  Roles, with mbarrier hand-offs instead of CTA
// barriers, so that copies, slicing, products and the epilogue of different
// chunks and block rows overlap:
//   warp 0 (one thread)   copies each chunk's window of x (8 rows x 32
//                         columns, one bulk copy per row; xr[s]) and then its
//                         image (full[s]) into a ring of kWsStages stages;
//   warps 2..7            cut the x window of each chunk into slices in the
//                         stage as soon as it has landed, while the image is
//                         still arriving (xfull[s]: all 192 threads have
//                         arrived); the phase of xr[s] also tells them that
//                         the stage's slices of the chunk kWsStages earlier
//                         have been consumed (the producer waited for that);
//   warp 1 (one thread)   issues the chunk's MMAs once both have arrived and
//                         commits them to empty[s] (the stage may be refilled)
//                         and, after a pass's last chunk, to accfull;
//   warps 8..15           read the accumulators of a finished pass, write r,
//                         and arrive on accempty, which the next pass's first
//                         MMA waits for (tensor memory holds one pass).
// Every wait is bounded and also ends when another role has given up
// (sAbort); the roles then stop, wait (bounded) for what they issued, and
// the kernel reports the error.
constexpr int kWsKC = 16;                                  // real K per chunk (8 complex columns)
constexpr int kWsChunks = 3 * 2 * 64 / kWsKC;              // 24 chunks per pass
constexpr int kWsASlice = kRtM * kWsKC * 2;                // 4096 bytes per matrix slice
constexpr int kWsAStage = kRtNSA * kWsASlice;              // 40960 bytes of matrix slices
constexpr int kWsBStage = kRtNSX * kRtNC * kWsKC * 2;      // 9216 bytes of x slices
constexpr int kWsXStage = 8 * kRtNC * 16;                  // 4096 bytes: the raw x window (complex128)
constexpr int kWsStage = kWsAStage + kWsBStage + kWsXStage;
constexpr int kWsStages = 4;
constexpr int kWsSlicers = 192, kWsEpi = 256;
static_assert(kWsChunks * kWsAStage == 12 * kRtAStage, "image bytes per block row");

// Byte offset of element (r, k) of a K-major, unswizzled tile of 16-bit
// elements 16 columns wide: core matrices of 8 rows x 8 elements, the two
// K-adjacent cores 128 bytes apart, 8-row groups 256 bytes apart.
__device__ __forceinline__ int kmajw(int r, int k) {
    return (r >> 3) * 256 + (k >> 3) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// The ten slices of matrix entry v (row i, complex column sl of a chunk, row
// exponent E) into the image tiles at dst, in the 16-wide layout.
__device__ __forceinline__ void slice_matrix_entry_w(z2 v, int E, int i, int sl, unsigned char *dst) {
    const unsigned long long qr = fixq<60>(v.x, E), qi = fixq<60>(v.y, E);
    const uint32_t sr = dsign(v.x), si = dsign(v.y);
    const uint32_t baser = 0x4B000000u | sr, basei = 0x4B000000u | si;
    const float offr = __uint_as_float(0xCB000000u ^ sr), offi = __uint_as_float(0xCB000000u ^ si);
    const int o_re = kmajw(i, 2 * sl), o_im = kmajw(i + 64, 2 * sl);
#pragma unroll
    for (int n = 0; n < kRtNSA; ++n) {
        const int sh = 54 - 6 * n;
        const uint32_t mr = (uint32_t)(qr >> sh) & 63u, mi = (uint32_t)(qi >> sh) & 63u;
        const uint32_t fr = f32_int(mr, baser, offr), fi = f32_int(mi, basei, offi);
        unsigned char *An = dst + n * kWsASlice;
        *reinterpret_cast<uint32_t *>(An + o_re) = bf16_pair(fr, fi ^ 0x80000000u);
        *reinterpret_cast<uint32_t *>(An + o_im) = bf16_pair(fi, fr);
    }
}

// Image (j, q) (block row j, chunk q = 8 b + c8: complex columns 8 c8 .. +7
// of block b of the coupling row): kWsAStage bytes.  Entry e of a chunk: row
// i = 8 (e >> 6) + ((e >> 2) & 7), column sl = 4 ((e >> 5) & 1) + (e & 3), so
// that a warp's 32 words are one contiguous 128-byte piece.
__global__ void __launch_bounds__(kRtThreads) k_matrix_image(ResidTcArgs a, unsigned char *img) {
    const int m = a.m;
    for (int64_t g = blockIdx.x; g < a.N * kWsChunks; g += gridDim.x) {
        const int64_t j = g / kWsChunks;
        const int q = (int)(g - j * kWsChunks), b = q >> 3, s0 = (q & 7) * 8;
        unsigned char *dst = img + g * (int64_t)kWsAStage;
        for (int e = threadIdx.x; e < 64 * 8; e += kRtThreads) {
            const int i = (e >> 6) * 8 + ((e >> 2) & 7), sl = ((e >> 5) & 1) * 4 + (e & 3);
            const int E = i < m ? a.erow[j * m + i] : kExpZero;
            slice_matrix_entry_w(coupling(a, j, b, i, s0 + sl), E, i, sl, dst);
        }
    }
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done)
                 : "r"(mbar), "r"(parity));
    return done != 0;
}

// Bounded wait that also gives up when another role has set *abort.
__device__ __forceinline__ bool wait_or_abort(uint32_t mbar, uint32_t parity, const volatile int *abort) {
    const long long t0 = clock64();
    for (int it = 0; it < kRtWaitPolls; ++it) {
        if (mbar_test(mbar, parity)) return true;
        if (*abort) return false;
        if (clock64() - t0 > 4000000000ll) break;
    }
    return false;
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__global__ void __launch_bounds__(kRtThreads, 1) k_residual_ws(ResidTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *full = reinterpret_cast<uint64_t *>(base + kWsStages * kWsStage);
    uint64_t *xfull = full + kWsStages, *empty = xfull + kWsStages;
    uint64_t *xr = empty + kWsStages;                     // [S] the x window of a stage has landed
    uint64_t *accfull = xr + kWsStages, *accempty = accfull + 1;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(accempty + 1);
    volatile int *sAbort = reinterpret_cast<volatile int *>(tmem_slot + 1);
    int *sEr = reinterpret_cast<int *>(tmem_slot + 4);          // [2][64]
    int *sEc = sEr + 128;                                        // [2][32]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m, k = a.k;
    const int64_t mk = (int64_t)m * k;
    const int npass = (k + kRtNC - 1) / kRtNC;
    const int64_t rows = a.N > blockIdx.x ? (a.N - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t passes = rows * npass, total = passes * kWsChunks;

    if (tid == 0) {
        for (int s = 0; s < kWsStages; ++s) {
            mbar_init(smem_u32(&full[s]), 1);
            mbar_init(smem_u32(&xfull[s]), kWsSlicers);
            mbar_init(smem_u32(&empty[s]), 1);
            mbar_init(smem_u32(&xr[s]), 1);
        }
        mbar_init(smem_u32(accfull), 1);
        mbar_init(smem_u32(accempty), kWsEpi);
        *sAbort = 0;
    }
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), kRtTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    auto stage = [&](int s) { return base + s * kWsStage; };
    auto row_of = [&](int64_t P) { return blockIdx.x + (P / npass) * (int64_t)gridDim.x; };

    if (warp == 0) {
        // producer: chunk images into the ring
        if (lane == 0) {
            int64_t G = 0;
            for (; G < total; ++G) {
                const int st = (int)(G % kWsStages);
                const uint32_t use = (uint32_t)(G / kWsStages);
                if (use > 0 && !wait_or_abort(smem_u32(&empty[st]), (use - 1) & 1u, sAbort)) break;
                const int64_t P = G / kWsChunks, j = row_of(P);
                const int c = (int)(G % kWsChunks), col0 = (int)(P % npass) * kRtNC;
                // the x window: rows s0 .. s0+7 of x_{j-1+b}, columns col0 .. col0+31
                const int b = c >> 3, s0 = (c & 7) * 8, nc = min(kRtNC, k - col0);
                const int64_t jb = j - 1 + b;
                const bool xin = jb >= 0 && jb < a.N;
                const int nr = xin ? max(0, min(8, m - s0)) : 0;
                uint32_t rowmask = 0;   // rows whose copy is issued (all of them outside bounds-checked builds)
                for (int r = 0; r < nr; ++r) {
                    const int64_t o = jb * mk + (int64_t)(s0 + r) * k + col0;
                    if (rin(a, kDbgResid, o) && rin(a, kDbgResid, o + nc - 1)) rowmask |= 1u << r;
                }
                // the x window first, on its own barrier, so that the slicers can
                // cut it while the image is still on its way
                mbar_expect_tx(smem_u32(&xr[st]), (uint32_t)(__popc(rowmask) * nc * 16));
                for (int r = 0; r < nr; ++r)
                    if (rowmask >> r & 1u)
                        bulk_g2s(smem_u32(stage(st) + kWsAStage + kWsBStage + r * kRtNC * 16),
                                 a.x + jb * mk + (int64_t)(s0 + r) * k + col0, (uint32_t)(nc * 16), smem_u32(&xr[st]));
                mbar_expect_tx(smem_u32(&full[st]), (uint32_t)kWsAStage);
                bulk_g2s(smem_u32(stage(st)), a.img + (j * kWsChunks + c) * (int64_t)kWsAStage, (uint32_t)kWsAStage,
                         smem_u32(&full[st]));
            }
            if (G < total) {
                *sAbort = 1;
                // the copies issued but not consumed must land before the CTA ends
                for (int64_t g = (G > kWsStages ? G - kWsStages : 0); g < G; ++g) {
                    mbar_wait(smem_u32(&xr[g % kWsStages]), (uint32_t)(g / kWsStages) & 1u, kRtWaitPolls);
                    mbar_wait(smem_u32(&full[g % kWsStages]), (uint32_t)(g / kWsStages) & 1u, kRtWaitPolls);
                }
            }
        }
    } else if (warp == 1) {
        // MMA issue
        if (lane == 0) {
            int64_t G = 0;
            bool ok = true;
            for (; G < total && ok; ++G) {
                const int st = (int)(G % kWsStages);
                const uint32_t use = (uint32_t)(G / kWsStages);
                const int64_t P = G / kWsChunks;
                const int c = (int)(G % kWsChunks);
                if (c == 0 && P > 0 && !wait_or_abort(smem_u32(accempty), (uint32_t)(P - 1) & 1u, sAbort)) break;
                if (!wait_or_abort(smem_u32(&full[st]), use & 1u, sAbort) ||
                    !wait_or_abort(smem_u32(&xfull[st]), use & 1u, sAbort)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t a0 = smem_u32(stage(st)), b0 = a0 + kWsAStage;
                const uint32_t acc = c == 0 ? 0u : 1u;
                const uint64_t bd = umma_desc(b0, 128, 256), bd8 = umma_desc(b0 + 8 * (kRtNC / 8) * 256, 128, 256);
                for (int i = 0; i < kRtNSA; ++i) {
                    const uint64_t ad = umma_desc(a0 + i * kWsASlice, 128, 256);
                    const int jmax = min(kRtNSX - 1, kRtND - 1 - i);
                    if (jmax == kRtNSX - 1) {
                        mma_bf16(tmem + i * kRtNC, ad, bd, idesc_bf16(kRtM, 256), i == 0 ? acc : 1u);
                        mma_bf16(tmem + (i + 8) * kRtNC, ad, bd8, idesc_bf16(kRtM, kRtNC), acc);
                    } else {
                        mma_bf16(tmem + i * kRtNC, ad, bd, idesc_bf16(kRtM, (jmax + 1) * kRtNC), 1u);
                    }
                }
                tc_commit(smem_u32(&empty[st]));
                if (c == kWsChunks - 1) tc_commit(smem_u32(accfull));
            }
            if (G < total) {
                *sAbort = 1;
                // the MMAs committed so far must finish before tensor memory is released
                if (G > 0) {
                    const int64_t g = G - 1;
                    mbar_wait(smem_u32(&empty[g % kWsStages]), (uint32_t)(g / kWsStages) & 1u, kRtWaitPolls);
                }
            }
        }
    } else if (warp < 8) {
        // x slicers: 192 threads, 256 entries (8 complex rows x 32 columns) per chunk
        const int sid = tid - 64;
        for (int64_t G = 0; G < total; ++G) {
            const int st = (int)(G % kWsStages);
            const uint32_t use = (uint32_t)(G / kWsStages);
            if (!wait_or_abort(smem_u32(&xr[st]), use & 1u, sAbort)) {
                *sAbort = 1;
                break;
            }
            const int64_t P = G / kWsChunks, j = row_of(P);
            const int c = (int)(G % kWsChunks), col0 = (int)(P % npass) * kRtNC, slot = (int)(P & 1);
            if (c == 0) {
                // the pass's exponents (its slot was last read by the epilogue of
                // pass P - 2, which ended before any MMA of pass P - 1)
                if (sid < 64) sEr[slot * 64 + sid] = sid < m ? a.erow[j * m + sid] : kExpZero;
                if (sid >= 64 && sid < 64 + kRtNC) {
                    const int cc = sid - 64, col = col0 + cc;
                    int F = kExpZero;
                    if (col < k) {
                        F = a.ecol[j * k + col];
                        if (j > 0) F = max(F, a.ecol[(j - 1) * k + col]);
                        if (j + 1 < a.N) F = max(F, a.ecol[(j + 1) * k + col]);
                    }
                    sEc[slot * 32 + cc] = F;
                }
                asm volatile("bar.sync 1, %0;" ::"n"(kWsSlicers) : "memory");
            }
            unsigned char *Bs = stage(st) + kWsAStage;
            const z2 *Xw = reinterpret_cast<const z2 *>(stage(st) + kWsAStage + kWsBStage);
            const int b = c >> 3, s0 = (c & 7) * 8;
            const int64_t jb = j - 1 + b;
            for (int e = sid; e < 8 * kRtNC; e += kWsSlicers) {
                const int sl = ((e >> 7) << 2) | (e & 3), cc = (((e >> 5) & 3) << 3) | ((e >> 2) & 7);
                const int s = s0 + sl, col = col0 + cc;
                z2 v = zmk(0.0, 0.0);
                if (s < m && col < k && jb >= 0 && jb < a.N) v = Xw[sl * kRtNC + cc];
                const int F = sEc[slot * 32 + cc];
                const unsigned long long qr = fixq<54>(v.x, F), qi = fixq<54>(v.y, F);
                const uint32_t sr = dsign(v.x), si = dsign(v.y);
                const uint32_t baser = 0x4B000000u | sr, basei = 0x4B000000u | si;
                const float offr = __uint_as_float(0xCB000000u ^ sr), offi = __uint_as_float(0xCB000000u ^ si);
                // the 54-bit integers as 30 high and 24 low bits: slices 0..4 from
                // the high word, 5..8 from the low one, each one 32-bit shift
                const uint32_t hr = (uint32_t)(qr >> 24), lr = (uint32_t)qr & 0xFFFFFFu;
                const uint32_t hi_ = (uint32_t)(qi >> 24), li = (uint32_t)qi & 0xFFFFFFu;
#pragma unroll
                for (int n = 0; n < kRtNSX; ++n) {
                    const int sh = n < 5 ? 24 - 6 * n : 18 - 6 * (n - 5);
                    const uint32_t mr = ((n < 5 ? hr : lr) >> sh) & 63u, mi = ((n < 5 ? hi_ : li) >> sh) & 63u;
                    *reinterpret_cast<uint32_t *>(Bs + kmajw(n * kRtNC + cc, 2 * sl)) =
                        bf16_pair(f32_int(mr, baser, offr), f32_int(mi, basei, offi));
                }
            }
            fence_async_smem();
            mbar_arrive(smem_u32(&xfull[st]));
        }
    } else {
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, columns 16 ((w - 8) / 4) .. +15
        const int p = (warp & 3) * 32 + lane, i = p & 63, part = p >> 6, half = (warp - 8) >> 2;
        // y of the thread's 4 columns of group g
        auto load_y = [&](int64_t j, int col0, int g, double (&yv)[4]) {
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int col = col0 + half * 16 + g * 4 + cc;
                const int64_t ro = (j * m + i) * (int64_t)k + col;
                yv[cc] = (a.y && i < m && col < k && rin(a, kDbgResid, ro))
                             ? __ldg(reinterpret_cast<const double *>(a.y + ro) + part)
                             : 0.0;
            }
        };
        for (int64_t P = 0; P < passes; ++P) {
            const int64_t j = row_of(P);
            const int col0 = (int)(P % npass) * kRtNC, slot = (int)(P & 1);
            if (!wait_or_abort(smem_u32(accfull), (uint32_t)P & 1u, sAbort)) {
                *sAbort = 1;
                break;
            }
            tc_fence_after();
            // The thread's 16 columns: T = sum_d acc_d 2^(6 (11 - d)), exact
            // (|T| < 2^91), as hi 2^36 + lo with hi = sum_{d<6} acc_d 2^(6 (5 - d))
            // and lo the rest (each below 2^55 in magnitude, so 64-bit), read
            // one diagonal (16 columns) at a time; tensor memory is released
            // right after, so that the next pass's products run while y - A x
            // is formed.
            long long hi[16], lo[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) hi[q] = lo[q] = 0;
#pragma unroll
            for (int d = 0; d < kRtND; ++d) {
                uint32_t v[16];
                tmem_ld16(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(d * kRtNC + half * 16), v);
                tmem_wait_ld();
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const long long x = __float2int_rn(__uint_as_float(v[q]));
                    if (d < 6) hi[q] = hi[q] * 64 + x;
                    else lo[q] = lo[q] * 64 + x;
                }
            }
            tc_fence_before();
            mbar_arrive(smem_u32(accempty));
            const int Er = sEr[slot * 64 + i];
#pragma unroll
            for (int g = 0; g < 4; ++g) {
                double ycur[4];
                load_y(j, col0, g, ycur);
#pragma unroll
                for (int cc = 0; cc < 4; ++cc) {
                    const int q = g * 4 + cc, c = half * 16 + q, col = col0 + c;
                    if (i >= m || col >= k) continue;
                    const int F = sEc[slot * 32 + c];
                    const __int128 T = (__int128)hi[q] * ((__int128)1 << 36) + (__int128)lo[q];
                    const int64_t ro = (j * m + i) * (int64_t)k + col;
                    if (!rin(a, kDbgResid, ro)) continue;
                    double *dst = &a.r[ro].x + part;
                    const double yv = ycur[cc];
                    double rv;
                    if (Er == kExpNonFinite || F == kExpNonFinite) {
                        rv = __longlong_as_double(0x7FF8000000000000ll);
                    } else if (Er == kExpZero || F == kExpZero) {
                        rv = yv;
                    } else if (!resid_exact(yv, T, Er + F - 76, rv)) {
                        rv = fma(-(double)T, pow2(Er + F - 76), yv);
                    }
                    *dst = rv;
                }
            }
        }
    }
    __syncthreads();
    if (*sAbort && tid == 0 && a.err) atomicExch(a.err, 1);
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kRtTmemCols);
}

// Without an image: every chunk's matrix slices are cut in the kernel (method
// CRSOLVE_RESIDUAL_SPLIT).
__global__ void __launch_bounds__(kRtThreads, 1) k_residual_tc(ResidTcArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    uint64_t *mbar = reinterpret_cast<uint64_t *>(base + 2 * kRtStage);   // [2] MMAs of a buffer done
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(base + 2 * kRtStage + 32);
    int *sEr = reinterpret_cast<int *>(base + 2 * kRtStage + 64);        // [64]
    int *sEc = sEr + 64;                                                  // [32]
    int *sAbort = sEc + kRtNC;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m = a.m, k = a.k;
    const int64_t mk = (int64_t)m * k;

    if (tid == 0) {
        mbar_init(smem_u32(&mbar[0]), 1);
        mbar_init(smem_u32(&mbar[1]), 1);
        *sAbort = 0;
    }
    if (warp == 0) tmem_alloc(smem_u32(tmem_slot), kRtTmemCols);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    uint32_t uses0 = 0, uses1 = 0;      // commits issued per buffer
    bool ok = true;
    const int npass = (k + kRtNC - 1) / kRtNC;

    // The raw FP64 values of the next chunk are loaded into registers while
    // the current one is cut into slices, so that the loads' latency hides
    // behind the integer work (and, across a pass boundary, behind the
    // epilogue).  Thread tid handles the matrix entries tid + u * 512 of a
    // chunk and x entry tid.
    constexpr int kAPer = (64 * 16) / kRtThreads;
    static_assert((64 * 16) % kRtThreads == 0 && 16 * kRtNC == kRtThreads, "one x entry per thread");
    z2 cur_a[kAPer], nxt_a[kAPer], cur_x, nxt_x;
    auto fetch = [&](int64_t jj, int c0, int q, z2 (&va)[kAPer], z2 &vx) {
        const int b = q >> 2, s0 = (q & 3) * 16;
#pragma unroll
        for (int u = 0; u < kAPer; ++u) {
            const int e = tid + u * kRtThreads;
            va[u] = coupling(a, jj, b, a_row(e), s0 + a_col(e));
        }
        const int s = s0 + x_row(tid), col = c0 + x_col(tid);
        const int64_t jb = jj - 1 + b;
        vx = zmk(0.0, 0.0);
        if (s < m && col < k && jb >= 0 && jb < a.N && rin(a, kDbgResid, jb * mk + (int64_t)s * k + col))
            vx = __ldg(a.x + jb * mk + (int64_t)s * k + col);
    };
    int64_t j = blockIdx.x;
    int pass = 0;
    if (j < a.N) fetch(j, 0, 0, cur_a, cur_x);
    while (j < a.N && ok) {
        const int col0 = pass * kRtNC;
        // the (row, pass) after this one: its first chunk is fetched during the last chunk
        int64_t jn = j;
        int pn = pass + 1;
        if (pn == npass) {
            pn = 0;
            jn = j + gridDim.x;
        }
        if (tid < 64) sEr[tid] = tid < m ? a.erow[j * m + tid] : kExpZero;
        if (tid >= 64 && tid < 64 + kRtNC) {
            const int c = tid - 64, col = col0 + c;
            int F = kExpZero;
            if (col < k) {
                F = a.ecol[j * k + col];
                if (j > 0) F = max(F, a.ecol[(j - 1) * k + col]);
                if (j + 1 < a.N) F = max(F, a.ecol[(j + 1) * k + col]);
            }
            sEc[c] = F;
        }
        __syncthreads();
        for (int q = 0; q < 12; ++q) {
            const int buf = (int)((uses0 + uses1) & 1u);
            const uint32_t ub = buf ? uses1 : uses0;
            // the buffer's previous MMAs must have read it
            if (ub > 0 && !mbar_wait(smem_u32(&mbar[buf]), (ub - 1) & 1u, kRtWaitPolls)) *sAbort = 1;
            __syncthreads();
            if (*sAbort) {
                ok = false;
                break;
            }
            unsigned char *As = base + buf * kRtStage, *Bs = As + kRtAStage;
            if (q + 1 < 12) fetch(j, col0, q + 1, nxt_a, nxt_x);
            else if (jn < a.N) fetch(jn, pn * kRtNC, 0, nxt_a, nxt_x);
            // matrix slices: 64 rows x 16 complex columns (see a_row / a_col
            // for the bank-conflict-free map)
#pragma unroll
            for (int u = 0; u < kAPer; ++u) {
                const int e = tid + u * kRtThreads, i = a_row(e), sl = a_col(e);
                slice_matrix_entry(cur_a[u], sEr[i], i, sl, As);
            }
            // x slices: 16 complex rows x 32 columns
            {
                const int c = x_col(tid), sl = x_row(tid);
                const z2 v = cur_x;
                const int F = sEc[c];
                const unsigned long long qr = fixq<54>(v.x, F), qi = fixq<54>(v.y, F);
                const uint32_t sr = dsign(v.x), si = dsign(v.y);
                const uint32_t baser = 0x4B000000u | sr, basei = 0x4B000000u | si;
                const float offr = __uint_as_float(0xCB000000u ^ sr), offi = __uint_as_float(0xCB000000u ^ si);
#pragma unroll
                for (int n = 0; n < kRtNSX; ++n) {
                    const int sh = 48 - 6 * n;
                    const uint32_t mr = (uint32_t)(qr >> sh) & 63u, mi = (uint32_t)(qi >> sh) & 63u;
                    *reinterpret_cast<uint32_t *>(Bs + kmaj16(n * kRtNC + c, 2 * sl)) =
                        bf16_pair(f32_int(mr, baser, offr), f32_int(mi, basei, offi));
                }
            }
#pragma unroll
            for (int u = 0; u < kAPer; ++u) cur_a[u] = nxt_a[u];
            cur_x = nxt_x;
            fence_async_smem();
            tc_fence_before();
            __syncthreads();
            tc_fence_after();
            if (tid == 0) {
                const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
                for (int t = 0; t < kRtKC / 16; ++t) {
                    // the first products of a pass start the accumulators
                    // (acc_0..acc_8 by slice 0, acc_9 by slice 1)
                    const uint32_t acc = (q == 0 && t == 0) ? 0u : 1u;
                    const uint64_t bd = umma_desc(b0 + t * 256, 128, 512);
                    const uint64_t bd8 = umma_desc(b0 + 8 * (kRtNC / 8) * 512 + t * 256, 128, 512);
                    for (int i = 0; i < kRtNSA; ++i) {
                        const uint64_t ad = umma_desc(a0 + i * kRtASlice + t * 256, 128, 512);
                        const int jmax = min(kRtNSX - 1, kRtND - 1 - i);
                        if (jmax == kRtNSX - 1) {
                            // x slices 0..7 (N = 256), then slice 8 (N = 32)
                            mma_bf16(tmem + i * kRtNC, ad, bd, idesc_bf16(kRtM, 256), i == 0 ? acc : 1u);
                            mma_bf16(tmem + (i + 8) * kRtNC, ad, bd8, idesc_bf16(kRtM, kRtNC), acc);
                        } else {
                            mma_bf16(tmem + i * kRtNC, ad, bd, idesc_bf16(kRtM, (jmax + 1) * kRtNC), 1u);
                        }
                    }
                }
                tc_commit(smem_u32(&mbar[buf]));
            }
            if (buf) ++uses1;
            else ++uses0;
        }
        if (!ok) break;
        // all MMAs of this pass: wait for the last commit (it tracks every earlier MMA)
        {
            const int lb = (int)((uses0 + uses1 - 1) & 1u);
            if (!mbar_wait(smem_u32(&mbar[lb]), ((lb ? uses1 : uses0) - 1) & 1u, kRtWaitPolls)) *sAbort = 1;
        }
        tc_fence_after();
        __syncthreads();
        if (*sAbort) {
            ok = false;
            break;
        }
        // epilogue: warp w reads TMEM lanes 32 (w % 4) .. +31, columns 8 (w / 4) .. +7
        const int p = (warp & 3) * 32 + lane, quarter = warp >> 2;
        const int i = p & 63, part = p >> 6;
        const int Er = sEr[i];
        for (int g = 0; g < 2; ++g) {
            const int cb = quarter * 8 + g * 4;
            uint32_t acc[kRtND][4];
#pragma unroll
            for (int d = 0; d < kRtND; ++d)
                tmem_ld4(tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)(d * kRtNC + cb), acc[d]);
            tmem_wait_ld();
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const int c = cb + cc, col = col0 + c;
                if (i >= m || col >= k) continue;
                const int F = sEc[c];
                // T = sum_d acc_d 2^(6 (11 - d)), exact (|T| < 2^91)
                __int128 T = 0;
#pragma unroll
                for (int d = 0; d < kRtND; ++d) T = T * 64 + (__int128)__float2int_rn(__uint_as_float(acc[d][cc]));
                const int64_t ro = (j * m + i) * (int64_t)k + col;
                if (!rin(a, kDbgResid, ro)) continue;
                double *dst = &a.r[ro].x + part;
                const double yv = a.y ? (&a.y[ro].x)[part] : 0.0;
                double rv;
                if (Er == kExpNonFinite || F == kExpNonFinite) {
                    rv = __longlong_as_double(0x7FF8000000000000ll);
                } else if (Er == kExpZero || F == kExpZero) {
                    rv = yv;
                } else if (!resid_exact(yv, T, Er + F - 76, rv)) {
                    rv = fma(-(double)T, pow2(Er + F - 76), yv);
                }
                *dst = rv;
            }
        }
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        j = jn;
        pass = pn;
    }
    if (!ok) {
        if (tid == 0 && a.err) atomicExch(a.err, 1);
        // let every committed MMA finish before tensor memory is released
        if (uses0 > 0) mbar_wait(smem_u32(&mbar[0]), (uses0 - 1) & 1u, kRtWaitPolls);
        if (uses1 > 0) mbar_wait(smem_u32(&mbar[1]), (uses1 - 1) & 1u, kRtWaitPolls);
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) tmem_dealloc(tmem, kRtTmemCols);
}

}  // namespace

size_t residual_tc_smem_bytes() { return 2 * (size_t)kRtStage + 1024 + 1024; }
static size_t residual_ws_smem_bytes() { return kWsStages * (size_t)kWsStage + 1024 + 1024; }

size_t residual_image_bytes(int64_t N) { return (size_t)N * kWsChunks * (size_t)kWsAStage; }

cudaError_t launch_matrix_image(const ResidTcArgs &a, unsigned char *img, int nsm, cudaStream_t s) {
    int64_t g = a.N * kWsChunks;
    if (g > (int64_t)nsm * 8) g = (int64_t)nsm * 8;
    k_matrix_image<<<(unsigned)g, kRtThreads, 0, s>>>(a, img);
    return cudaGetLastError();
}

cudaError_t launch_row_exponents(const ResidTcArgs &a, int nsm, cudaStream_t s) {
    const int64_t n = a.N * a.m;
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)nsm * 16) g = (int64_t)nsm * 16;
    k_row_exponents<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_residual_tc(const ResidTcArgs &a, int nsm, cudaStream_t s) {
    const int64_t n = a.N * a.k;
    int64_t g = (n + 255) / 256;
    if (g > (int64_t)nsm * 16) g = (int64_t)nsm * 16;
    k_col_exponents<<<(unsigned)(g < 1 ? 1 : g), 256, 0, s>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = residual_tc_smem_bytes();
    const int64_t grid = a.N < nsm ? a.N : nsm;
    if (a.img) {
        const size_t wsm = residual_ws_smem_bytes();
        e = cudaFuncSetAttribute(k_residual_ws, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)wsm);
        if (e != cudaSuccess) return e;
        k_residual_ws<<<(unsigned)grid, kRtThreads, wsm, s>>>(a);
    } else {
        e = cudaFuncSetAttribute(k_residual_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_residual_tc<<<(unsigned)grid, kRtThreads, smem, s>>>(a);
    }
    return cudaGetLastError();
}

}  // namespace crs

// ---------------------------------------------------------------- C ABI

namespace {

size_t split_ws_bytes(int64_t N, int m, int k, bool image) {
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    return up(256) + up((size_t)N * m * sizeof(int)) + up((size_t)N * k * sizeof(int)) +
           (image ? up(crs::residual_image_bytes(N)) : 0);
}

}  // namespace

extern "C" int crsolve_residual_workspace_bytes(int64_t N, int32_t m, int32_t k, int32_t method, size_t *bytes) {
    if (!bytes || N < 1 || m < 1 || k < 1) return CRSOLVE_EINVAL;
    if (m > CRSOLVE_MAX_M || k > CRSOLVE_MAX_K) return CRSOLVE_EUNSUPPORTED;
    if (method == CRSOLVE_RESIDUAL_FP64) {
        *bytes = 0;
        return CRSOLVE_OK;
    }
    if (method != CRSOLVE_RESIDUAL_SPLIT && method != CRSOLVE_RESIDUAL_SPLIT_IMAGE) return CRSOLVE_EUNSUPPORTED;
    *bytes = split_ws_bytes(N, m, k, method == CRSOLVE_RESIDUAL_SPLIT_IMAGE);
    return CRSOLVE_OK;
}

extern "C" int crsolve_residual(int64_t N, int32_t m, int32_t k, const crsolve_z *A, const crsolve_z *B,
                                const crsolve_z *x, const crsolve_z *y, crsolve_z *r, int32_t method,
                                void *workspace, size_t workspace_bytes, void *stream) {
    if (N < 1 || m < 1 || k < 1 || !A || !x || !y || !r || (N > 1 && !B)) return CRSOLVE_EINVAL;
    if (m > CRSOLVE_MAX_M || k > CRSOLVE_MAX_K) return CRSOLVE_EUNSUPPORTED;
    if ((((uintptr_t)A | (uintptr_t)B | (uintptr_t)x | (uintptr_t)y | (uintptr_t)r) & 15u) ||
        (const void *)r == (const void *)x)
        return CRSOLVE_EINVAL;
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return CRSOLVE_ECUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    using crs::z2;
    if (method == CRSOLVE_RESIDUAL_FP64)
        return crs::launch_residual(N, m, k, reinterpret_cast<const z2 *>(A), reinterpret_cast<const z2 *>(B),
                                    reinterpret_cast<const z2 *>(x), reinterpret_cast<const z2 *>(y),
                                    reinterpret_cast<z2 *>(r), nsm, s) == cudaSuccess
                   ? CRSOLVE_OK
                   : CRSOLVE_ECUDA;
    if (method != CRSOLVE_RESIDUAL_SPLIT && method != CRSOLVE_RESIDUAL_SPLIT_IMAGE) return CRSOLVE_EUNSUPPORTED;
    const bool image = method == CRSOLVE_RESIDUAL_SPLIT_IMAGE;
    if (!workspace || workspace_bytes < split_ws_bytes(N, m, k, image) || ((uintptr_t)workspace & 255u))
        return CRSOLVE_EINVAL;
    char *ws = static_cast<char *>(workspace);
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    crs::ResidTcArgs a{};
    a.N = N; a.m = m; a.k = k;
    a.A = reinterpret_cast<const z2 *>(A);
    a.B = reinterpret_cast<const z2 *>(B);
    a.x = reinterpret_cast<const z2 *>(x);
    a.y = reinterpret_cast<const z2 *>(y);
    a.r = reinterpret_cast<z2 *>(r);
    a.err = reinterpret_cast<int *>(ws);
    a.erow = reinterpret_cast<int *>(ws + up(256));
    a.ecol = reinterpret_cast<int *>(ws + up(256) + up((size_t)N * m * sizeof(int)));
    if (cudaMemsetAsync(a.err, 0, sizeof(int), s) != cudaSuccess) return CRSOLVE_ECUDA;
    if (crs::launch_row_exponents(a, nsm, s) != cudaSuccess) return CRSOLVE_ECUDA;
    if (image) {
        unsigned char *img = reinterpret_cast<unsigned char *>(
            ws + up(256) + up((size_t)N * m * sizeof(int)) + up((size_t)N * k * sizeof(int)));
        if (crs::launch_matrix_image(a, img, nsm, s) != cudaSuccess) return CRSOLVE_ECUDA;
        a.img = img;
    }
    if (crs::launch_residual_tc(a, nsm, s) != cudaSuccess) return CRSOLVE_ECUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, a.err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    return err ? CRSOLVE_ETIMEOUT : CRSOLVE_OK;
}
