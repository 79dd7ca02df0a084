// cr_levels.cu -- the per-level kernels of classic cyclic reduction in FP64
// (one chunk of odd blocks per CTA; the steps themselves are in cr_core.cuh)
// and their host-side launchers.
#include "cr_launch.h"
#include "cr_core.cuh"

namespace crs {

template <int MT, class R>
__global__ void __launch_bounds__(256) k_factor_odd(LevelArgsT<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    factor_chunk<MT, R>(a, a.c_begin + blockIdx.x, smem_raw);
}

// The FP32 factor of class MT = 64 (tensor-core Schur product, L^{-1}): its
// shared memory allows one CTA per SM, so the registers may be spent freely.
__global__ void __launch_bounds__(256, 1) k_factor_odd_f32_64(LevelArgsT<float> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    factor_chunk<64, float>(a, a.c_begin + blockIdx.x, smem_raw);
}

template <class R>
__global__ void __launch_bounds__(256) k_factor_fix(LevelArgsT<R> a) {
    factor_fix_items<R>(a, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

template <int MT, class R>
__global__ void __launch_bounds__(256) k_solve_down_odd(LevelArgsT<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    solve_down_chunk<MT, R>(a, a.c_begin + blockIdx.x, blockIdx.y, smem_raw);
}

template <class R>
__global__ void __launch_bounds__(256) k_solve_down_fix(LevelArgsT<R> a) {
    solve_down_fix_items<R>(a, blockIdx.x * (int64_t)blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
}

template <int MT, class R>
__global__ void __launch_bounds__(256) k_solve_up(LevelArgsT<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    solve_up_chunk<MT, R>(a, a.c_begin + blockIdx.x, blockIdx.y, smem_raw);
}

// The FP64 sweeps of class 16 at the default 128 threads, with registers
// capped so that five CTAs fit on an SM (16 warps otherwise): more warps to
// cover the loads at the start of each chunk.
__global__ void __launch_bounds__(128, 5) k_solve_down_odd_16c(LevelArgsT<double> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    solve_down_chunk<16, double>(a, a.c_begin + blockIdx.x, blockIdx.y, smem_raw);
}
__global__ void __launch_bounds__(128, 5) k_solve_up_16c(LevelArgsT<double> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    solve_up_chunk<16, double>(a, a.c_begin + blockIdx.x, blockIdx.y, smem_raw);
}

// The wide forms of the class MT < 32 (right-looking Cholesky, substitutions
// by (block, row, column) items; see trsv_lower_wide) for the coarse levels.
// Separate instances, so that the column-per-thread kernels keep their
// register allocation.
template <int MT, class R>
__global__ void __launch_bounds__(256) k_factor_odd_wide(LevelArgsT<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    factor_chunk<MT, R, true>(a, a.c_begin + blockIdx.x, smem_raw);
}
template <int MT, class R>
__global__ void __launch_bounds__(256) k_solve_down_odd_wide(LevelArgsT<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    solve_down_chunk<MT, R, true>(a, a.c_begin + blockIdx.x, blockIdx.y, smem_raw);
}
template <int MT, class R>
__global__ void __launch_bounds__(256) k_solve_up_wide(LevelArgsT<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    solve_up_chunk<MT, R, true>(a, a.c_begin + blockIdx.x, blockIdx.y, smem_raw);
}

// ------------------------------------------------------------------ adjoint

// gA_j = -1/2 (gy_j x_j^H + x_j gy_j^H) (lower, mirrored), and
// gB_j = -(gy_{j+1} x_j^H + x_{j+1} gy_j^H).
__global__ void __launch_bounds__(256) k_adjoint_outer(int64_t N, int m, int k, const z2 *__restrict__ x,
                                                        const z2 *__restrict__ gy, z2 *gA, z2 *gB) {
    const int mm = m * m, nl = m * (m + 1) / 2;
    const int64_t mk = (int64_t)m * k;
    const int64_t nA = gA ? N * nl : 0, nB = gB ? (N - 1) * mm : 0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nA + nB;
         e += (int64_t)gridDim.x * blockDim.x) {
        if (e < nA) {
            const int64_t j = e / nl;
            const int f = (int)(e - j * nl);
            const int p = tri_row(f), q = f - p * (p + 1) / 2;
            const z2 *g = gy + j * mk, *xx = x + j * mk;
            z2 acc = zmk(0.0, 0.0);
            for (int c = 0; c < k; ++c) {
                zmac_ca(acc, xx[q * k + c], g[p * k + c]);   // gy_p conj(x_q)
                zmac_ca(acc, g[q * k + c], xx[p * k + c]);   // x_p conj(gy_q)
            }
            acc = zscale(acc, -0.5);
            if (p == q) acc.y = 0.0;
            gA[j * mm + p * m + q] = acc;
            if (p != q) gA[j * mm + q * m + p] = zconj(acc);
        } else {
            const int64_t e2 = e - nA, j = e2 / mm;
            const int f = (int)(e2 - j * mm), p = f / m, q = f - p * m;
            const z2 *g0 = gy + j * mk, *g1 = gy + (j + 1) * mk, *x0 = x + j * mk, *x1 = x + (j + 1) * mk;
            z2 acc = zmk(0.0, 0.0);
            for (int c = 0; c < k; ++c) {
                zmac_ca(acc, x0[q * k + c], g1[p * k + c]);  // gy_{j+1,p} conj(x_{j,q})
                zmac_ca(acc, g0[q * k + c], x1[p * k + c]);  // x_{j+1,p} conj(gy_{j,q})
            }
            gB[j * mm + p * m + q] = zneg(acc);
        }
    }
}

__global__ void k_nan_if_failed(z2 *x, int64_t n, const unsigned long long *status) {
    if (*status == CRS_NO_FAIL) return;
    const z2 nan2 = zmk(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        x[e] = nan2;
}

// ------------------------------------------------------------- host side

// Default tile shapes per block-size class (swept on a GB300: N = 2^20,
// m = 8, k = 4; N = 2^16, m = 16, k = 8; N = 2^12, m = 32, k = 16;
// N = 2^14, m = 64, k = 32); crsolve_tile_set overrides them.
static TileShape g_tiles[5] = {
    {32, 32, 32, 256, 256},  // MT = 4
    {16, 16, 16, 256, 256},  // MT = 8
    {8, 4, 8, 256, 128},     // MT = 16
    {2, 1, 16, 256, 256},    // MT = 32
    {1, 1, 16, 256, 256},    // MT = 64
};

static int mt_slot(int mt) {
    switch (mt) {
        case 4: return 0;
        case 8: return 1;
        case 16: return 2;
        case 32: return 3;
        case 64: return 4;
        default: return -1;
    }
}

TileShape tile_shape(int mt) {
    const int i = mt_slot(mt);
    return i < 0 ? TileShape{0, 0, 0, 0, 0} : g_tiles[i];
}

// FP32 levels of the mixed-precision form: narrower right-hand-side chunks at
// MT >= 32 so that the staged Z still leaves room for two CTAs per SM.
static TileShape g_tiles32[5] = {
    {32, 32, 32, 256, 256}, {16, 16, 16, 256, 256}, {4, 8, 16, 256, 256}, {2, 2, 16, 256, 256},
    {1, 1, 16, 256, 256},
};

TileShape tile_shape32(int mt) {
    const int i = mt_slot(mt);
    return i < 0 ? TileShape{0, 0, 0, 0, 0} : g_tiles32[i];
}

bool set_tile_shape32(int mt, const TileShape &ts, size_t smem_limit) {
    const int i = mt_slot(mt);
    if (i < 0 || ts.nb_factor < 1 || ts.nb_solve < 1 || ts.kc_max < 1 || ts.threads < 32 ||
        ts.threads > 256 || ts.threads % 32 || ts.threads_solve < 32 || ts.threads_solve > 256 ||
        ts.threads_solve % 32)
        return false;
    // the FP32 factor of MT = 64 (blocked, tensor-core Schur product) has
    // its work split for exactly 256 threads
    if (mt == 64 && ts.threads != 256) return false;
    // (the solve fields are not used at MT = 64: see solve_nb32)
    if (factor_smem_bytes(mt, ts.nb_factor, 4) > smem_limit ||
        (mt != 64 && solve_smem_bytes(mt, ts.nb_solve, ts.kc_max, 3, 4) > smem_limit))
        return false;
    g_tiles32[i] = ts;
    return true;
}

bool set_tile_shape(int mt, const TileShape &ts, size_t smem_limit) {
    const int i = mt_slot(mt);
    if (i < 0 || ts.nb_factor < 1 || ts.nb_solve < 1 || ts.kc_max < 1 || ts.threads < 32 ||
        ts.threads > 256 || ts.threads % 32 || ts.threads_solve < 32 || ts.threads_solve > 256 ||
        ts.threads_solve % 32)
        return false;
    if (factor_smem_bytes(mt, ts.nb_factor, 8) > smem_limit ||
        solve_smem_bytes(mt, ts.nb_solve, ts.kc_max, 3, 8) > smem_limit)
        return false;
    g_tiles[i] = ts;
    return true;
}

int pick_mt(int m) {
    if (m <= 4) return 4;
    if (m <= 8) return 8;
    if (m <= 16) return 16;
    if (m <= 32) return 32;
    if (m <= 64) return 64;
    return 0;
}

// Per block: packed L (later P^H P) and packed V, Z = [P | Q], 1/diag(L);
// rsize = bytes of the real type (8 for FP64, 4 for FP32).
size_t factor_smem_bytes(int mt, int nb, int rsize) {
    const size_t tri = (size_t)mt * (mt + 1) / 2, cs = 2 * (size_t)rsize;
    size_t b = (size_t)nb * ((2 * tri + 2 * (size_t)mt * mt) * cs + (size_t)mt * rsize);
    if (rsize == 4 && mt == 64) {
        b += 1024 + tc_stage_bytes(mt);                 // tensor-core operand stages (1 KB aligned)
        b += (size_t)nb * mt * kF32LdE * cs;             // L^{-1} of every block (padded rows)
    }
    return b;
}

// Per block: packed L, `panels` right-hand-side panels of MT x kc (3 down, 3 up), 1/diag(L),
// and for FP32 with MT >= 32 the staged Z [MT][2MT] (after 8 bytes of alignment padding).
size_t solve_smem_bytes(int mt, int nb, int kc, int panels, int rsize) {
    const size_t tri = (size_t)mt * (mt + 1) / 2, cs = 2 * (size_t)rsize;
    size_t b = (size_t)nb * (tri * cs + (size_t)mt * kc * cs * panels + (size_t)mt * rsize);
    if (rsize == 4 && mt >= 32) b += 8 + (size_t)nb * mt * 2 * mt * cs;
    return b;
}

// Allow every kernel the device's full opt-in shared memory, so that any
// tile shape that set_tile_shape accepted can launch.
template <int MT, class R>
static cudaError_t prepare_mt_r(int smem_optin) {
    cudaError_t e;
    e = cudaFuncSetAttribute(k_factor_odd<MT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
    if (e != cudaSuccess) return e;
    if constexpr (MT == 64 && sizeof(R) == 4) {
        e = cudaFuncSetAttribute(k_factor_odd_f32_64, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
    }
    if constexpr (MT == 16 && sizeof(R) == 8) {
        e = cudaFuncSetAttribute(k_solve_down_odd_16c, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_solve_up_16c, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
    }
    if constexpr (MT < 32) {
        e = cudaFuncSetAttribute(k_factor_odd_wide<MT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_solve_down_odd_wide<MT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 smem_optin);
        if (e != cudaSuccess) return e;
        e = cudaFuncSetAttribute(k_solve_up_wide<MT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
        if (e != cudaSuccess) return e;
    }
    e = cudaFuncSetAttribute(k_solve_down_odd<MT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_solve_up<MT, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
}

template <int MT>
static cudaError_t prepare_mt(int smem_optin) {
    const cudaError_t e = prepare_mt_r<MT, double>(smem_optin);
    return e != cudaSuccess ? e : prepare_mt_r<MT, float>(smem_optin);
}

cudaError_t prepare_kernels(int mt) {
    int dev = 0, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return e;
    switch (mt) {
        case 4: return prepare_mt<4>(optin);
        case 8: return prepare_mt<8>(optin);
        case 16: return prepare_mt<16>(optin);
        case 32: return prepare_mt<32>(optin);
        case 64: {
            const cudaError_t e2 = prepare_mt<64>(optin);
            return e2 != cudaSuccess ? e2 : prepare_solve_g32(optin);
        }
        default: return cudaErrorInvalidValue;
    }
}

static int level_nb(int nb_max, int64_t no, int nsm) {
    int64_t want = (no + 2 * (int64_t)nsm - 1) / (2 * (int64_t)nsm);
    if (want < 1) want = 1;
    return (int)(want < nb_max ? want : nb_max);
}

int factor_nb(int mt, int64_t no, int nsm) { return level_nb(tile_shape(mt).nb_factor, no, nsm); }
int solve_nb(int mt, int64_t no, int nsm) { return level_nb(tile_shape(mt).nb_solve, no, nsm); }
// Right-hand-side columns per solve CTA: the tile's chunk, narrowed on levels
// with few odd blocks so that the column chunks still spread over about two
// CTAs per SM (the columns of a triangular solve are independent).
static int spread_kc(int kmax, int k, int64_t ncta_blocks, int nsm) {
    int kc = k < kmax ? k : kmax;
    const int64_t want = 2 * (int64_t)nsm;
    if (ncta_blocks * ((k + kc - 1) / kc) < want) {
        const int64_t chunks = (want + ncta_blocks - 1) / ncta_blocks;
        int64_t c = (k + chunks - 1) / chunks;
        if (c < 1) c = 1;
        if (c < kc) kc = (int)c;
    }
    return kc;
}

int solve_kc(int mt, int k, int64_t no, int nsm) {
    return spread_kc(tile_shape(mt).kc_max, k, num_ctas(no, solve_nb(mt, no, nsm)), nsm);
}
int factor_nb32(int mt, int64_t no, int nsm) { return level_nb(tile_shape32(mt).nb_factor, no, nsm); }
// MT = 64: one odd block per work item of the persistent product kernels
// (cr_solve32.cu), whose column chunk depends on k alone.
int solve_nb32(int mt, int64_t no, int nsm) { return mt == 64 ? 1 : level_nb(tile_shape32(mt).nb_solve, no, nsm); }
int solve_kc32(int mt, int k, int64_t no, int nsm) {
    if (mt == 64) {
        // levels with fewer work items than SMs: narrower column chunks, so
        // that the items of a level spread over more SMs
        int kc = solve_kc_g32(k);
        while (kc > 8 && no * ((k + kc - 1) / kc) < nsm) kc /= 2;
        return kc;
    }
    return spread_kc(tile_shape32(mt).kc_max, k, num_ctas(no, solve_nb32(mt, no, nsm)), nsm);
}

// CTAs of one launch of an odd-block kernel: the chunk range, else the level.
template <class R>
static unsigned odd_grid(const LevelArgsT<R> &a) {
    return (unsigned)(a.c_count > 0 ? a.c_count : num_ctas(a.no, a.nb));
}

static unsigned grid_1d(int64_t items, int nsm) {
    int64_t g = (items + 255) / 256;
    const int64_t cap = (int64_t)nsm * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

// The wide kernels of the class MT < 32 serve the levels that the tile was
// narrowed for (fewer blocks or columns per CTA than the tile's: the coarse
// levels, about two CTAs per SM) when a CTA holds at most kWideCols
// substitution columns, i.e. when a column per thread would keep at most two
// warps of the CTA busy.  Their results are bit-identical.
constexpr int kWideCols = 64;

template <int MT, class R>
static bool factor_wide(const LevelArgsT<R> &a) {
    const TileShape ts = sizeof(R) == 4 ? tile_shape32(MT) : tile_shape(MT);
    return MT < 32 && a.nb < ts.nb_factor && a.nb * 2 * a.m <= kWideCols;
}

template <int MT, class R>
static bool solve_wide(const LevelArgsT<R> &a) {
    const TileShape ts = sizeof(R) == 4 ? tile_shape32(MT) : tile_shape(MT);
    const bool narrowed = a.nb < ts.nb_solve || a.kc < (a.k < ts.kc_max ? a.k : ts.kc_max);
    return MT < 32 && narrowed && a.nb * a.kc <= kWideCols;
}

template <int MT, class R>
static cudaError_t factor_odd_mt(const LevelArgsT<R> &a, cudaStream_t s) {
    const unsigned grid = odd_grid(a);
    const int th = sizeof(R) == 4 ? tile_shape32(MT).threads : tile_shape(MT).threads;
    if constexpr (MT == 64 && sizeof(R) == 4) {
        k_factor_odd_f32_64<<<grid, th, factor_smem_bytes(MT, a.nb, sizeof(R)), s>>>(a);
    } else if constexpr (MT < 32) {
        if (factor_wide<MT, R>(a))
            k_factor_odd_wide<MT, R><<<grid, th, factor_smem_bytes(MT, a.nb, sizeof(R)), s>>>(a);
        else
            k_factor_odd<MT, R><<<grid, th, factor_smem_bytes(MT, a.nb, sizeof(R)), s>>>(a);
    } else {
        k_factor_odd<MT, R><<<grid, th, factor_smem_bytes(MT, a.nb, sizeof(R)), s>>>(a);
    }
    return cudaGetLastError();
}

template <int MT, class R>
static cudaError_t solve_down_odd_mt(const LevelArgsT<R> &a, cudaStream_t s) {
    const dim3 grid(odd_grid(a), (unsigned)((a.k + a.kc - 1) / a.kc));
    const int th = sizeof(R) == 4 ? tile_shape32(MT).threads_solve : tile_shape(MT).threads_solve;
    if constexpr (MT < 32) {
        if (solve_wide<MT, R>(a)) {
            k_solve_down_odd_wide<MT, R><<<grid, th, solve_smem_bytes(MT, a.nb, a.kc, 3, sizeof(R)), s>>>(a);
            return cudaGetLastError();
        }
    }
    if constexpr (MT == 16 && sizeof(R) == 8) {
        if (th == 128) {
            k_solve_down_odd_16c<<<grid, th, solve_smem_bytes(MT, a.nb, a.kc, 3, sizeof(R)), s>>>(a);
            return cudaGetLastError();
        }
    }
    k_solve_down_odd<MT, R><<<grid, th, solve_smem_bytes(MT, a.nb, a.kc, 3, sizeof(R)), s>>>(a);
    return cudaGetLastError();
}

template <int MT, class R>
static cudaError_t solve_up_mt(const LevelArgsT<R> &a, cudaStream_t s) {
    const dim3 grid(odd_grid(a), (unsigned)((a.k + a.kc - 1) / a.kc));
    const int th = sizeof(R) == 4 ? tile_shape32(MT).threads_solve : tile_shape(MT).threads_solve;
    if constexpr (MT < 32) {
        if (solve_wide<MT, R>(a)) {
            k_solve_up_wide<MT, R><<<grid, th, solve_smem_bytes(MT, a.nb, a.kc, 3, sizeof(R)), s>>>(a);
            return cudaGetLastError();
        }
    }
    if constexpr (MT == 16 && sizeof(R) == 8) {
        if (th == 128) {
            k_solve_up_16c<<<grid, th, solve_smem_bytes(MT, a.nb, a.kc, 3, sizeof(R)), s>>>(a);
            return cudaGetLastError();
        }
    }
    k_solve_up<MT, R><<<grid, th, solve_smem_bytes(MT, a.nb, a.kc, 3, sizeof(R)), s>>>(a);
    return cudaGetLastError();
}

#define CRS_DISPATCH(fn, R, mt, ...)                 \
    switch (mt) {                                    \
        case 4: return fn<4, R>(__VA_ARGS__);        \
        case 8: return fn<8, R>(__VA_ARGS__);        \
        case 16: return fn<16, R>(__VA_ARGS__);      \
        case 32: return fn<32, R>(__VA_ARGS__);      \
        case 64: return fn<64, R>(__VA_ARGS__);      \
        default: return cudaErrorInvalidValue;       \
    }

template <class R>
static cudaError_t factor_fix_r(const LevelArgsT<R> &a, int nsm, cudaStream_t s) {
    const int64_t nbd = a.c_count > 0 ? a.c_count : num_ctas(a.no, a.nb) - 1;
    if (nbd < 1) return cudaSuccess;
    k_factor_fix<R><<<grid_1d(nbd * (a.m * (a.m + 1) / 2), nsm), 256, 0, s>>>(a);
    return cudaGetLastError();
}

template <class R>
static cudaError_t solve_down_fix_r(const LevelArgsT<R> &a, int nsm, cudaStream_t s) {
    const int64_t ncta = num_ctas(a.no, a.nb);
    if (ncta < 2) return cudaSuccess;
    k_solve_down_fix<R><<<grid_1d((ncta - 1) * a.m * a.k, nsm), 256, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_factor_odd(int mt, const LevelArgsT<double> &a, cudaStream_t s) {
    CRS_DISPATCH(factor_odd_mt, double, mt, a, s)
}
cudaError_t launch_factor_odd(int mt, const LevelArgsT<float> &a, cudaStream_t s) {
    CRS_DISPATCH(factor_odd_mt, float, mt, a, s)
}
cudaError_t launch_factor_fix(const LevelArgsT<double> &a, int nsm, cudaStream_t s) { return factor_fix_r(a, nsm, s); }
cudaError_t launch_factor_fix(const LevelArgsT<float> &a, int nsm, cudaStream_t s) { return factor_fix_r(a, nsm, s); }
cudaError_t launch_solve_down_odd(int mt, const LevelArgsT<double> &a, cudaStream_t s) {
    CRS_DISPATCH(solve_down_odd_mt, double, mt, a, s)
}
cudaError_t launch_solve_down_odd(int mt, const LevelArgsT<float> &a, cudaStream_t s) {
    if (mt == 64) return launch_solve_down_g32(a, s);   // L^{-1} form (cr_solve32.cu)
    CRS_DISPATCH(solve_down_odd_mt, float, mt, a, s)
}
cudaError_t launch_solve_down_fix(const LevelArgsT<double> &a, int nsm, cudaStream_t s) {
    return solve_down_fix_r(a, nsm, s);
}
cudaError_t launch_solve_down_fix(const LevelArgsT<float> &a, int nsm, cudaStream_t s) {
    return solve_down_fix_r(a, nsm, s);
}
cudaError_t launch_solve_up(int mt, const LevelArgsT<double> &a, cudaStream_t s) {
    CRS_DISPATCH(solve_up_mt, double, mt, a, s)
}
cudaError_t launch_solve_up(int mt, const LevelArgsT<float> &a, cudaStream_t s) {
    if (mt == 64) return launch_solve_up_g32(a, s);
    CRS_DISPATCH(solve_up_mt, float, mt, a, s)
}

cudaError_t launch_adjoint_outer(int64_t N, int m, int k, const z2 *x, const z2 *gy, z2 *gA, z2 *gB,
                                 int nsm, cudaStream_t s) {
    const int64_t items = (gA ? N * (m * (m + 1) / 2) : 0) + (gB ? (N - 1) * m * m : 0);
    if (items == 0) return cudaSuccess;
    k_adjoint_outer<<<grid_1d(items, nsm), 256, 0, s>>>(N, m, k, x, gy, gA, gB);
    return cudaGetLastError();
}

cudaError_t launch_nan_if_failed(z2 *x, int64_t n, const unsigned long long *status, int nsm,
                                 cudaStream_t s) {
    k_nan_if_failed<<<grid_1d(n, nsm), 256, 0, s>>>(x, n, status);
    return cudaGetLastError();
}

}  // namespace crs
