// crsolve_noalloc.cu -- crsolve_solve_noalloc: factor and solve one system
// without allocating device memory.
//
// Some callers cannot call cudaMalloc: code that runs where the allocator is
// not available or not allowed (for example inside a host callback, in a
// pre-allocated real-time loop, or from a plugin that must not grow the
// process's device footprint after start-up).  For them every intermediate of
// the cyclic reduction (the per-level factors, the reduced systems, the
// CTA-boundary buffers and the breakdown status) lives in one fixed array of
// this library, g_noalloc_scratch, of kNoAllocScratchBytes (32 MiB).  Every
// GPU that loads the library holds that array until the process exits.
//
// Rules for callers:
//   - Every call looks up the array's device address with
//     cudaGetSymbolAddress, with the caller's device current, and raises the
//     shared-memory limits of the kernels it launches.  Nothing is cached
//     between calls, so the address is never stale (after cudaDeviceReset, or
//     under another context of the same device).  The first call on a device
//     also loads the library's kernels onto it: make that first call before
//     any stream capture.
//   - All calls share the array and it keeps the last call's contents: calls
//     whose work overlaps on the GPU (different streams, or different host
//     threads on one device) race.  Serialise them.
//   - A system whose intermediates do not fit in the array is rejected with
//     CRSOLVE_ENOMEM before anything is launched.
#include <cstdint>

#include "crsolve.h"
#include "cr_launch.h"

using crs::z2;

namespace {

constexpr size_t kNoAllocScratchBytes = size_t(32) << 20;
constexpr int kMaxLevels = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

struct NaLevel {
    int64_t Nl, no, ne;
    size_t offL, offInv, offZ, offR, offAn, offBn, offYn, offXn;
};

size_t bump(size_t &cursor, size_t bytes) {
    const size_t off = cursor;
    cursor += (bytes + 255) & ~(size_t)255;
    return off;
}

}  // namespace

extern "C" int crsolve_solve_noalloc(int64_t N, int32_t m, int32_t k, const crsolve_z *A, const crsolve_z *B,
                                     const crsolve_z *y, crsolve_z *x, crsolve_info *info, void *stream) {
    if (N < 1 || m < 1 || k < 1 || !A || !y || !x || (N > 1 && !B)) return CRSOLVE_EINVAL;
    if (m > CRSOLVE_MAX_M || k > CRSOLVE_MAX_K) return CRSOLVE_EUNSUPPORTED;
    if ((((uintptr_t)A | (uintptr_t)y | (uintptr_t)x | (uintptr_t)B) & 15u) || (const void *)x == (const void *)y)
        return CRSOLVE_EINVAL;

    // The level-0 factors and the level-1 system alone take N complex m x m
    // blocks, so a larger N cannot fit.  Rejecting it first keeps every size
    // product below from overflowing (and the breakdown record's 40-bit block
    // index exact).
    if ((uint64_t)N > kNoAllocScratchBytes / ((size_t)m * m * sizeof(crsolve_z)) || (uint64_t)N >= (1ull << 40))
        return CRSOLVE_ENOMEM;
    // level schedule and the layout of the fixed array (no heap, no device allocation)
    NaLevel lev[kMaxLevels];
    int nlev = 0;
    const size_t zsz = sizeof(crsolve_z), mm = (size_t)m * m, mk = (size_t)m * k;
    size_t cur = 0;
    const size_t offStatus = bump(cur, 256);
    const size_t offDbg = bump(cur, 256);
    for (int64_t Nl = N;; Nl /= 2) {
        NaLevel &L = lev[nlev++];
        L.Nl = Nl; L.no = (Nl + 1) / 2; L.ne = Nl / 2;
        L.offL = bump(cur, L.no * mm * zsz);
        L.offInv = bump(cur, L.no * (size_t)m * sizeof(double));
        L.offZ = bump(cur, L.no * 2 * mm * zsz);
        L.offR = bump(cur, L.no * mk * zsz);
        L.offAn = bump(cur, L.ne * mm * zsz);
        L.offBn = bump(cur, (L.ne > 1 ? L.ne - 1 : 0) * mm * zsz);
        L.offYn = bump(cur, L.ne * mk * zsz);
        L.offXn = bump(cur, L.ne * mk * zsz);
        if (Nl == 1 || nlev == kMaxLevels) break;
    }
    const int64_t no0 = (N + 1) / 2;
    const size_t offWbd = bump(cur, no0 * mm * zsz);
    const size_t offCbd = bump(cur, no0 * mk * zsz);
    if (cur > kNoAllocScratchBytes) return CRSOLVE_ENOMEM;

    int dev = -1, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) return CRSOLVE_ECUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return CRSOLVE_ECUDA;
    const int mt = crs::pick_mt(m);
    // Set-up, with the caller's device current: the device address of the
    // array (in host code g_noalloc_scratch names a host-side stand-in, not
    // device memory) and the kernels' shared-memory limits.
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return CRSOLVE_ECUDA;
    if (crs::prepare_kernels(mt) != cudaSuccess) return CRSOLVE_ECUDA;
    char *ws = static_cast<char *>(p);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    unsigned long long *status = reinterpret_cast<unsigned long long *>(ws + offStatus);
    unsigned long long *dbg = reinterpret_cast<unsigned long long *>(ws + offDbg);
    // the array keeps the previous call's contents: the status must start as "no breakdown"
    if (cudaMemsetAsync(status, 0xFF, sizeof(unsigned long long), s) != cudaSuccess) return CRSOLVE_ECUDA;
#ifdef CRSOLVE_DEBUG_BOUNDS
    if (cudaMemsetAsync(dbg, 0xFF, sizeof(unsigned long long), s) != cudaSuccess) return CRSOLVE_ECUDA;
#endif

    auto args = [&](int l) {
        crs::LevelArgs a{};
        const NaLevel &L = lev[l];
        a.Nl = L.Nl; a.no = L.no; a.ne = L.ne; a.m = m; a.k = k; a.level = l;
        a.A = l == 0 ? reinterpret_cast<const z2 *>(A) : reinterpret_cast<const z2 *>(ws + lev[l - 1].offAn);
        a.B = l == 0 ? reinterpret_cast<const z2 *>(B) : reinterpret_cast<const z2 *>(ws + lev[l - 1].offBn);
        a.L = reinterpret_cast<z2 *>(ws + L.offL);
        a.inv = reinterpret_cast<double *>(ws + L.offInv);
        a.Z = reinterpret_cast<z2 *>(ws + L.offZ);
        a.Wbd = reinterpret_cast<z2 *>(ws + offWbd);
        a.An = reinterpret_cast<z2 *>(ws + L.offAn);
        a.Bn = reinterpret_cast<z2 *>(ws + L.offBn);
        a.y = l == 0 ? reinterpret_cast<const z2 *>(y) : reinterpret_cast<const z2 *>(ws + lev[l - 1].offYn);
        a.r = reinterpret_cast<z2 *>(ws + L.offR);
        a.cbd = reinterpret_cast<z2 *>(ws + offCbd);
        a.yn = reinterpret_cast<z2 *>(ws + L.offYn);
        a.xn = reinterpret_cast<const z2 *>(ws + L.offXn);
        a.x = l == 0 ? reinterpret_cast<z2 *>(x) : reinterpret_cast<z2 *>(ws + lev[l - 1].offXn);
        a.status = status;
        a.dbg = dbg;
        return a;
    };
    for (int l = 0; l < nlev; ++l) {
        crs::LevelArgs a = args(l);
        a.nb = crs::factor_nb(mt, a.no, nsm);
        if (crs::launch_factor_odd(mt, a, s) != cudaSuccess) return CRSOLVE_ECUDA;
        if (crs::num_ctas(a.no, a.nb) > 1 && crs::launch_factor_fix(a, nsm, s) != cudaSuccess) return CRSOLVE_ECUDA;
    }
    for (int l = 0; l < nlev; ++l) {
        crs::LevelArgs a = args(l);
        a.nb = crs::solve_nb(mt, a.no, nsm);
        a.kc = crs::solve_kc(mt, k, a.no, nsm);
        if (crs::launch_solve_down_odd(mt, a, s) != cudaSuccess) return CRSOLVE_ECUDA;
        if (crs::num_ctas(a.no, a.nb) > 1 && crs::launch_solve_down_fix(a, nsm, s) != cudaSuccess)
            return CRSOLVE_ECUDA;
    }
    for (int l = nlev - 1; l >= 0; --l) {
        crs::LevelArgs a = args(l);
        a.nb = crs::solve_nb(mt, a.no, nsm);
        a.kc = crs::solve_kc(mt, k, a.no, nsm);
        if (crs::launch_solve_up(mt, a, s) != cudaSuccess) return CRSOLVE_ECUDA;
    }
    if (info) {
        unsigned long long st = 0;
        if (cudaMemcpyAsync(&st, status, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess) return CRSOLVE_ECUDA;
        if (cudaStreamSynchronize(s) != cudaSuccess) return CRSOLVE_ECUDA;
        if (st == CRS_NO_FAIL) {
            *info = crsolve_info{CRSOLVE_OK, 0, 0, 0};
        } else {
            const int level = (int)(st >> 40);
            const int64_t block = (int64_t)(st & ((1ull << 40) - 1));
            *info = crsolve_info{CRSOLVE_NOT_PD, level, block, block << level};
        }
    }
    return CRSOLVE_OK;
}
