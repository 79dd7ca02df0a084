// crsolve_api.cu -- the C ABI declared in include/crsolve.h: plans, the
// workspace layout, and the level schedule of classic cyclic reduction.
//
// Level schedule: N_0 = N, N_{l+1} = floor(N_l / 2), down to N_L = 1.  Level l
// has ceil(N_l/2) odd blocks (factored and eliminated) and floor(N_l/2) even
// blocks (the next level).  Every block row of the original system is an odd
// block at exactly one level, so the factorisation does N block Cholesky
// factorisations in total.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "crsolve.h"
#include "cr_launch.h"

using crs::z2;

namespace {

struct LevelPlan {
    int64_t Nl, no, ne;
    size_t offL, offInv, offZ;       // stored factor of the odd blocks
    size_t offAn, offBn;             // next level system (l + 1)
    size_t offR, offYn, offXn;       // solve: r of this level, y and x of level l + 1
};

// Mixed precision: levels below `lT` run in FP32 (their own layout), the
// coarsest levels (N_l <= kMixedCoarse blocks: the last two) and the
// refinement in FP64.
constexpr int64_t kMixedCoarse = 2;
constexpr int kMixedMaxIter = 40;

// Workspace offsets with this bit set address the plan's scratch buffer
// (plans split by crsolve_plan_keep_levels); the others the workspace.
constexpr size_t kScr = size_t(1) << 62;

struct WsMap {
    char *ws, *scr;
    char *operator+(size_t off) const { return (off & kScr) ? scr + (off & ~kScr) : ws + off; }
};

}  // namespace

struct crsolve_plan_s {
    int64_t N = 0;
    int m = 0, kmax = 0, precision = 0, mt = 0, device = 0, nsm = 0;
    uint32_t flags = 0;
    std::vector<LevelPlan> lev;
    size_t offStatus = 0, offDbg = 0, offWbd = 0, offCbd = 0;
    // arrival counters of the chunk boundaries (bd_arrive): one per CTA of the
    // largest level and right-hand-side column, bdc_cap of them (0: none)
    size_t offBdc = 0;
    int64_t bdc_cap = 0;
    size_t offSA = 0, offSB = 0, offSY = 0, offSX = 0;
    size_t total = 0;
    char *ws = nullptr;
    size_t ws_bytes = 0;
    // keep_levels split (keep >= 0): factors of levels < keep and the level-keep
    // system in the workspace; coarser factors, solve buffers and CTA-boundary
    // scratch in the scratch buffer, whose coarse factors are rebuilt from the
    // level-keep system after the scratch has been (re)bound
    int keep = -1;
    char *scr = nullptr;
    size_t scr_total = 0;
    bool coarse_valid = false;
    const z2 *lvl0A = nullptr, *lvl0B = nullptr;   // the caller's A, B (re-factor from level 0)
    WsMap map() const { return WsMap{ws, scr}; }
    bool factored = false;
    bool prepared = false;
    // mixed precision
    int lT = 0;                                  // first FP64 level
    std::vector<LevelPlan> lev32;                // FP32 layout of levels < lT
    size_t offWbd32 = 0, offCbd32 = 0, offA32 = 0, offB32 = 0, offY32 = 0, offX32 = 0, offR64 = 0, offNorms = 0,
           offErr = 0;
    size_t offP64 = 0, offW64 = 0, offDot = 0, offScal = 0, offErow = 0, offEcol = 0;   // conjugate gradients
    size_t offAimg = 0;                                                                   // residual's matrix slices
    const crsolve_z *A64 = nullptr, *B64 = nullptr;  // the caller's FP64 system, read by the residual
    bool fallback = false;                       // FP32 factor broke down: everything in FP64
    int last_iters = 0;
    double last_delta = 0.0, last_rho = 0.0;
    // Algorithm 1 (CRSOLVE_PLAN_ALG1): levels 0..aL (aL = log2 N, the last
    // one being the single blocks), two reductions per level: alev[0] reads
    // the level buffer from block 1 (the concatenation of the split systems),
    // alev[1] from block 0 (the same, behind the auxiliary block A_0 = I)
    bool alg1 = false;
    int aL = 0;
    std::vector<LevelPlan> alev[2];
    size_t offA1A[2] = {0, 0}, offA1B[2] = {0, 0}, offA1Y[2] = {0, 0}, offA1R[2] = {0, 0};
    size_t offA1Xb = 0, offA1Xz = 0;
    // crsolve_solve_host: a copy stream (created on first use) and its events
    cudaStream_t cstream = nullptr;
    std::vector<cudaEvent_t> xev;
    // instrumentation
    bool timing = false;
    struct Rec { int kind, level; int64_t units; cudaEvent_t e0, e1; };
    std::vector<Rec> recs;
    std::vector<cudaEvent_t> pool;
    size_t pool_used = 0;
    int64_t launches = 0;
};

namespace {

// NVTX range for the lifetime of the object (tracing with Nsight tools;
// near-free when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    NvtxRange(const char *what, int level) {
        char buf[48];
        snprintf(buf, sizeof buf, "%s level %d", what, level);
        nvtxRangePushA(buf);
    }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

size_t take(size_t &cursor, size_t bytes) {
    const size_t off = cursor;
    cursor += (bytes + 255) & ~(size_t)255;
    return off;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

crs::LevelArgs level_args(const crsolve_plan_s *p, int l, const z2 *A0, const z2 *B0) {
    const LevelPlan &L = p->lev[l];
    crs::LevelArgs a{};
    a.Nl = L.Nl; a.no = L.no; a.ne = L.ne;
    a.m = p->m; a.level = l;
    const WsMap ws = p->map();
    a.A = (l == 0) ? A0 : reinterpret_cast<const z2 *>(ws + p->lev[l - 1].offAn);
    a.B = (l == 0) ? B0 : reinterpret_cast<const z2 *>(ws + p->lev[l - 1].offBn);
    a.L = reinterpret_cast<z2 *>(ws + L.offL);
    a.inv = reinterpret_cast<double *>(ws + L.offInv);
    a.Z = reinterpret_cast<z2 *>(ws + L.offZ);
    a.Wbd = reinterpret_cast<z2 *>(ws + p->offWbd);
    a.An = reinterpret_cast<z2 *>(ws + L.offAn);
    a.Bn = reinterpret_cast<z2 *>(ws + L.offBn);
    a.r = reinterpret_cast<z2 *>(ws + L.offR);
    a.cbd = reinterpret_cast<z2 *>(ws + p->offCbd);
    a.yn = reinterpret_cast<z2 *>(ws + L.offYn);
    a.xn = reinterpret_cast<const z2 *>(ws + L.offXn);
    a.status = reinterpret_cast<unsigned long long *>(ws + p->offStatus);
    a.dbg = reinterpret_cast<unsigned long long *>(ws + p->offDbg);
    return a;
}

crs::LevelArgsT<float> level_args32(const crsolve_plan_s *p, int l) {
    const LevelPlan &L = p->lev32[l];
    crs::LevelArgsT<float> a{};
    a.Nl = L.Nl; a.no = L.no; a.ne = L.ne;
    a.m = p->m; a.level = l;
    const WsMap ws = p->map();
    using C = crs::c2;
    a.A = reinterpret_cast<const C *>(ws + (l == 0 ? p->offA32 : p->lev32[l - 1].offAn));
    a.B = reinterpret_cast<const C *>(ws + (l == 0 ? p->offB32 : p->lev32[l - 1].offBn));
    a.L = reinterpret_cast<C *>(ws + L.offL);
    a.inv = reinterpret_cast<float *>(ws + L.offInv);
    a.Z = reinterpret_cast<C *>(ws + L.offZ);
    a.Wbd = reinterpret_cast<C *>(ws + p->offWbd32);
    a.An = reinterpret_cast<C *>(ws + L.offAn);
    a.Bn = reinterpret_cast<C *>(ws + L.offBn);
    a.r = reinterpret_cast<C *>(ws + L.offR);
    a.cbd = reinterpret_cast<C *>(ws + p->offCbd32);
    a.yn = reinterpret_cast<C *>(ws + L.offYn);
    a.xn = reinterpret_cast<const C *>(ws + L.offXn);
    a.y = reinterpret_cast<const C *>(ws + (l == 0 ? p->offY32 : p->lev32[l - 1].offYn));
    a.x = reinterpret_cast<C *>(ws + (l == 0 ? p->offX32 : p->lev32[l - 1].offXn));
    a.status = reinterpret_cast<unsigned long long *>(ws + p->offStatus);
    a.err = reinterpret_cast<int *>(ws + p->offErr);
    a.dbg = reinterpret_cast<unsigned long long *>(ws + p->offDbg);
    return a;
}

// The mixed form's residuals by exact splitting on the tensor cores (m > 32,
// unless the plan asks for the FP64 pipe).
bool mixed_uses_split(const crsolve_plan_s *p) { return p->m > 32 && !(p->flags & CRSOLVE_PLAN_FP64_RESIDUAL); }

// Bounds-checked builds: clear the plan's out-of-range record (all ones =
// none) before a factorisation; release builds enqueue nothing.
int debug_reset(crsolve_plan_s *p, cudaStream_t s) {
#ifdef CRSOLVE_DEBUG_BOUNDS
    if (cudaMemsetAsync(p->ws + p->offDbg, 0xFF, sizeof(unsigned long long), s) != cudaSuccess) return CRSOLVE_ECUDA;
#else
    (void)p;
    (void)s;
#endif
    return CRSOLVE_OK;
}

int ensure_prepared(crsolve_plan_s *p) {
    if (p->prepared) return CRSOLVE_OK;
    if (crs::prepare_kernels(p->mt) != cudaSuccess) return CRSOLVE_ECUDA;
    p->prepared = true;
    return CRSOLVE_OK;
}

int check_device(const crsolve_plan_s *p) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return CRSOLVE_ECUDA;
    return dev == p->device ? CRSOLVE_OK : CRSOLVE_EINVAL;
}

cudaEvent_t next_event(crsolve_plan_s *p) {
    if (p->pool_used == p->pool.size()) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        p->pool.push_back(e);
    }
    return p->pool[p->pool_used++];
}

// Launch one kernel through fn(), counting it and, when timing is on,
// bracketing it with events on stream s.
template <class F>
int launch(crsolve_plan_s *p, int kind, int level, int64_t units, cudaStream_t s, F &&fn) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (p->timing) {
        e0 = next_event(p);
        e1 = next_event(p);
        if (!e0 || !e1 || cudaEventRecord(e0, s) != cudaSuccess) return CRSOLVE_ECUDA;
    }
    if (fn() != cudaSuccess) return CRSOLVE_ECUDA;
    p->launches += 1;
    if (p->timing) {
        if (cudaEventRecord(e1, s) != cudaSuccess) return CRSOLVE_ECUDA;
        p->recs.push_back({kind, level, units, e0, e1});
    }
    return CRSOLVE_OK;
}

// ---- Algorithm 1 -----------------------------------------------------------
//
// Level l of Algorithm 1 (Sec. 3) holds 2^l split systems of n = N/2^l
// blocks.  They are stored one after another as one block-tridiagonal system
// of N blocks, with zero couplings across system boundaries, behind one
// auxiliary block (A = I, B = 0, y = 0) at buffer position 0.  One level is
// then two classic reductions of the same buffer:
//   h = 0: from block 1 (the concatenation); it eliminates the odd blocks of
//          every split system, and its even system is, block for block, the
//          concatenation of their even halves (V, F, v of eq. Formulas);
//   h = 1: from block 0 (the concatenation shifted by one); it eliminates the
//          auxiliary block and the even blocks, and its even system is the
//          concatenation of the odd halves (U, E, u).
// A zero coupling stays exactly zero through a reduction (P = L^{-1} 0), so
// the split systems stay decoupled.  The next level stores the odd halves at
// positions 1..N/2 and the even halves at N/2+1..N, with the coupling between
// them (position N/2 of the B buffer) zero.  Position p of level l therefore
// holds original block rotl^l(p) (on log2 N bits), and after log2 N levels
// the single blocks are back in the original order.  The last level (single
// blocks, every coupling zero) is factored and solved by the same two
// reductions, whose back-substitution then reduces to x = L^{-H} L^{-1} y.
crs::LevelArgs alg1_args(const crsolve_plan_s *p, int l, int h) {
    const LevelPlan &H = p->alev[h][l];
    crs::LevelArgs a{};
    a.Nl = H.Nl; a.no = H.no; a.ne = H.ne;
    a.m = p->m; a.level = l;
    const int64_t N = p->N, in0 = (h == 0) ? 1 : 0, out0 = (h == 0) ? 1 + N / 2 : 1;
    const size_t mm = (size_t)p->m * p->m;
    const int cur = l & 1, nxt = cur ^ 1;
    const WsMap ws = p->map();
    a.A = reinterpret_cast<const z2 *>(ws + p->offA1A[cur]) + in0 * mm;
    a.B = reinterpret_cast<const z2 *>(ws + p->offA1B[cur]) + in0 * mm;
    a.An = reinterpret_cast<z2 *>(ws + p->offA1A[nxt]) + out0 * mm;
    a.Bn = reinterpret_cast<z2 *>(ws + p->offA1B[nxt]) + out0 * mm;
    a.L = reinterpret_cast<z2 *>(ws + H.offL);
    a.inv = reinterpret_cast<double *>(ws + H.offInv);
    a.Z = reinterpret_cast<z2 *>(ws + H.offZ);
    a.Wbd = reinterpret_cast<z2 *>(ws + p->offWbd);
    a.r = reinterpret_cast<z2 *>(ws + p->offA1R[h]);
    a.cbd = reinterpret_cast<z2 *>(ws + p->offCbd);
    a.status = reinterpret_cast<unsigned long long *>(ws + p->offStatus);
    a.rep_bits = p->aL;
    a.rep_off = (h == 0) ? 0 : -1;
    return a;
}

int alg1_factor(crsolve_plan_s *p, const z2 *A, const z2 *B, cudaStream_t s) {
    const int64_t N = p->N;
    const size_t mm = (size_t)p->m * p->m, zsz = sizeof(z2);
    z2 *A0 = reinterpret_cast<z2 *>(p->map() + p->offA1A[0]), *A1 = reinterpret_cast<z2 *>(p->map() + p->offA1A[1]);
    z2 *B0 = reinterpret_cast<z2 *>(p->map() + p->offA1B[0]), *B1 = reinterpret_cast<z2 *>(p->map() + p->offA1B[1]);
    if (cudaMemsetAsync(p->map() + p->offStatus, 0xFF, sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMemcpyAsync(A0 + mm, A, N * mm * zsz, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        (N > 1 && cudaMemcpyAsync(B0 + mm, B, (N - 1) * mm * zsz, cudaMemcpyDeviceToDevice, s) != cudaSuccess))
        return CRSOLVE_ECUDA;
    int rc;
    if ((rc = launch(p, CRSOLVE_K_ALG1_BORDER, 0, 1, s, [&] {
             return crs::launch_alg1_border(A0, A1, B0, B1, N > 1 ? B1 + (N / 2) * mm : nullptr, p->m, s);
         })))
        return rc;
    for (int l = 0; l <= p->aL; ++l) {
        for (int h = 1; h >= 0; --h) {
            if (h == 1 && N < 2) continue;
            crs::LevelArgs a = alg1_args(p, l, h);
            a.nb = crs::factor_nb(p->mt, a.no, p->nsm);
            if ((rc = launch(p, CRSOLVE_K_FACTOR_ODD, l, a.no, s,
                             [&] { return crs::launch_factor_odd(p->mt, a, s); })))
                return rc;
            if (crs::num_ctas(a.no, a.nb) > 1 &&
                (rc = launch(p, CRSOLVE_K_FACTOR_FIX, l, crs::num_ctas(a.no, a.nb) - 1, s,
                             [&] { return crs::launch_factor_fix(a, p->nsm, s); })))
                return rc;
        }
        // buffer 0 held the caller's coupling at position N/2; from level 2 on it
        // is the (zero) coupling between the odd and the even halves
        if (l == 0 && p->aL >= 2 && cudaMemsetAsync(B0 + (N / 2) * mm, 0, mm * zsz, s) != cudaSuccess)
            return CRSOLVE_ECUDA;
    }
    p->factored = true;
    return CRSOLVE_OK;
}

int alg1_solve(crsolve_plan_s *p, int k, const z2 *y, z2 *x, cudaStream_t s) {
    const int64_t N = p->N;
    const size_t mk = (size_t)p->m * k, zsz = sizeof(z2);
    z2 *Y[2] = {reinterpret_cast<z2 *>(p->map() + p->offA1Y[0]), reinterpret_cast<z2 *>(p->map() + p->offA1Y[1])};
    z2 *Xb = reinterpret_cast<z2 *>(p->map() + p->offA1Xb), *Xz = reinterpret_cast<z2 *>(p->map() + p->offA1Xz);
    if (cudaMemcpyAsync(Y[0] + mk, y, N * mk * zsz, cudaMemcpyDeviceToDevice, s) != cudaSuccess ||
        cudaMemsetAsync(Y[0], 0, mk * zsz, s) != cudaSuccess || cudaMemsetAsync(Y[1], 0, mk * zsz, s) != cudaSuccess ||
        cudaMemsetAsync(Xz, 0, (N / 2 + 1) * mk * zsz, s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    int rc;
    for (int l = 0; l <= p->aL; ++l) {
        const int cur = l & 1, nxt = cur ^ 1;
        for (int h = 1; h >= 0; --h) {
            if (h == 1 && N < 2) continue;
            crs::LevelArgs a = alg1_args(p, l, h);
            a.k = k;
            a.nb = crs::solve_nb(p->mt, a.no, p->nsm);
            a.kc = crs::solve_kc(p->mt, k, a.no, p->nsm);
            a.y = Y[cur] + ((h == 0) ? 1 : 0) * mk;
            a.yn = Y[nxt] + ((h == 0) ? 1 + N / 2 : 1) * mk;
            if ((rc = launch(p, CRSOLVE_K_SOLVE_DOWN_ODD, l, a.no, s,
                             [&] { return crs::launch_solve_down_odd(p->mt, a, s); })))
                return rc;
            if (crs::num_ctas(a.no, a.nb) > 1 &&
                (rc = launch(p, CRSOLVE_K_SOLVE_DOWN_FIX, l, crs::num_ctas(a.no, a.nb) - 1, s,
                             [&] { return crs::launch_solve_down_fix(a, p->nsm, s); })))
                return rc;
        }
    }
    // single blocks: x = L^{-H} r of both reductions (zero even unknowns and
    // couplings), from block 1 straight into x, the shifted one into Xb
    for (int h = 0; h < 2; ++h) {
        if (h == 1 && N < 2) continue;
        crs::LevelArgs a = alg1_args(p, p->aL, h);
        a.k = k;
        a.nb = crs::solve_nb(p->mt, a.no, p->nsm);
        a.kc = crs::solve_kc(p->mt, k, a.no, p->nsm);
        a.xn = Xz;
        a.x = (h == 0) ? x : Xb;
        if ((rc = launch(p, CRSOLVE_K_SOLVE_UP, p->aL, a.no, s,
                         [&] { return crs::launch_solve_up(p->mt, a, s); })))
            return rc;
    }
    if (N >= 2 && (rc = launch(p, CRSOLVE_K_ALG1_MERGE, p->aL, N, s, [&] {
                       return crs::launch_alg1_merge(x, Xb, N, (int64_t)mk,
                                                     reinterpret_cast<const unsigned long long *>(p->map() + p->offStatus),
                                                     p->nsm, s);
                   })))
        return rc;
    return CRSOLVE_OK;
}

// CTA-boundary completion inside the odd-block kernels (bd_arrive) pays on
// the coarse levels, where a fix-up launch costs more than the level's
// work; on the fine levels the fence and atomics at the end of every one of
// their many short CTAs cost about as much as the fix-up kernel (measured:
// k_solve_down_odd +0.16 ms per step at N = 2^20, m = 8), so launches of
// more than kBdMaxCtasPerSm CTAs per SM keep the fix-up kernel.
constexpr int64_t kBdMaxCtasPerSm = 4;
bool fuse_boundaries(const crsolve_plan_s *p, int64_t ctas) { return ctas <= kBdMaxCtasPerSm * p->nsm; }

// Arrival counters for launches that need `need` of them (zeroed on the
// stream), or nullptr when the plan's region is too small (the levels then
// take the fix-up kernels).
unsigned *boundary_counters(crsolve_plan_s *p, int64_t need, cudaStream_t s, int *rc) {
    *rc = CRSOLVE_OK;
    if (need < 1 || need > p->bdc_cap) return nullptr;
    unsigned *cnt = reinterpret_cast<unsigned *>(p->map() + p->offBdc);
    if (cudaMemsetAsync(cnt, 0, (size_t)need * sizeof(unsigned), s) != cudaSuccess) *rc = CRSOLVE_ECUDA;
    return cnt;
}

// Factor levels [l0, nlev): the odd-block kernel per level, which also
// completes the CTA-boundary even blocks (bd_arrive), or else a fix-up
// kernel after it.
int factor_levels(crsolve_plan_s *p, int l0, const z2 *A, const z2 *B, cudaStream_t s) {
    int rc;
    int64_t need = 0;
    for (int l = l0; l < (int)p->lev.size(); ++l) {
        const int64_t ctas = crs::num_ctas(p->lev[l].no, crs::factor_nb(p->mt, p->lev[l].no, p->nsm));
        if (fuse_boundaries(p, ctas)) need = std::max(need, ctas);
    }
    unsigned *cnt = boundary_counters(p, need, s, &rc);
    if (rc) return rc;
    for (int l = l0; l < (int)p->lev.size(); ++l) {
        NvtxRange nv("factor", l);
        crs::LevelArgs a = level_args(p, l, A, B);
        a.nb = crs::factor_nb(p->mt, a.no, p->nsm);
        a.bd_count = fuse_boundaries(p, crs::num_ctas(a.no, a.nb)) ? cnt : nullptr;
        if ((rc = launch(p, CRSOLVE_K_FACTOR_ODD, l, a.no, s,
                         [&] { return crs::launch_factor_odd(p->mt, a, s); })))
            return rc;
        if (!a.bd_count && crs::num_ctas(a.no, a.nb) > 1 &&
            (rc = launch(p, CRSOLVE_K_FACTOR_FIX, l, crs::num_ctas(a.no, a.nb) - 1, s,
                         [&] { return crs::launch_factor_fix(a, p->nsm, s); })))
            return rc;
    }
    return CRSOLVE_OK;
}

int do_factor(crsolve_plan_s *p, const z2 *A, const z2 *B, cudaStream_t s) {
    if (p->alg1) return alg1_factor(p, A, B, s);
    if (cudaMemsetAsync(p->map() + p->offStatus, 0xFF, sizeof(unsigned long long), s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    int rc;
    if ((rc = factor_levels(p, 0, A, B, s))) return rc;
    p->factored = true;
    return CRSOLVE_OK;
}

crs::LevelArgs solve_args(const crsolve_plan_s *p, int l, int k) {
    crs::LevelArgs a = level_args(p, l, nullptr, nullptr);
    a.k = k;
    a.nb = crs::solve_nb(p->mt, a.no, p->nsm);
    a.kc = crs::solve_kc(p->mt, k, a.no, p->nsm);
    return a;
}

// Down sweep of every level, then the up sweep of levels nlev-1 .. l_end.
int solve_sweeps(crsolve_plan_s *p, int k, const z2 *y, z2 *x, int l_end, cudaStream_t s) {
    const int nlev = (int)p->lev.size();
    int rc;
    // the down sweep completes its CTA-boundary right-hand sides itself
    // (bd_arrive; counters per CTA and column chunk) or takes fix-up kernels
    int64_t need = 0;
    auto ctas_of = [&](const crs::LevelArgs &a) { return crs::num_ctas(a.no, a.nb) * ((k + a.kc - 1) / a.kc); };
    for (int l = 0; l < nlev; ++l) {
        const int64_t ctas = ctas_of(solve_args(p, l, k));
        if (fuse_boundaries(p, ctas)) need = std::max(need, ctas);
    }
    unsigned *cnt = boundary_counters(p, need, s, &rc);
    if (rc) return rc;
    for (int l = 0; l < nlev; ++l) {
        NvtxRange nv("solve down", l);
        crs::LevelArgs a = solve_args(p, l, k);
        a.y = (l == 0) ? y : reinterpret_cast<const z2 *>(p->map() + p->lev[l - 1].offYn);
        a.bd_count = fuse_boundaries(p, ctas_of(a)) ? cnt : nullptr;
        if ((rc = launch(p, CRSOLVE_K_SOLVE_DOWN_ODD, l, a.no, s,
                         [&] { return crs::launch_solve_down_odd(p->mt, a, s); })))
            return rc;
        if (!a.bd_count && crs::num_ctas(a.no, a.nb) > 1 &&
            (rc = launch(p, CRSOLVE_K_SOLVE_DOWN_FIX, l, crs::num_ctas(a.no, a.nb) - 1, s,
                         [&] { return crs::launch_solve_down_fix(a, p->nsm, s); })))
            return rc;
    }
    for (int l = nlev - 1; l >= l_end; --l) {
        NvtxRange nv("solve up", l);
        crs::LevelArgs a = solve_args(p, l, k);
        a.x = (l == 0) ? x : reinterpret_cast<z2 *>(p->map() + p->lev[l - 1].offXn);
        if ((rc = launch(p, CRSOLVE_K_SOLVE_UP, l, a.no, s,
                         [&] { return crs::launch_solve_up(p->mt, a, s); })))
            return rc;
    }
    return CRSOLVE_OK;
}

int do_solve(crsolve_plan_s *p, int k, const z2 *y, z2 *x, cudaStream_t s) {
    if (p->alg1) return alg1_solve(p, k, y, x, s);
    return solve_sweeps(p, k, y, x, 0, s);
}

// Plans split by crsolve_plan_keep_levels: after the scratch has been (re)bound
// the factors of levels keep .. L are rebuilt from the level-keep system kept
// in the workspace (for keep = 0: the caller's A, B), the recursion of Sec. 2
// restarted at level keep.  Deterministic, so they equal the lost ones.
int ensure_coarse(crsolve_plan_s *p, cudaStream_t s) {
    if (p->keep < 0 || p->coarse_valid) return CRSOLVE_OK;
    if (!p->scr) return CRSOLVE_ENOMEM;
    if (p->keep == 0 && !p->lvl0A) return CRSOLVE_ENOTFACTORED;
    int rc;
    if ((rc = factor_levels(p, p->keep, p->lvl0A, p->lvl0B, s))) return rc;
    p->coarse_valid = true;
    return CRSOLVE_OK;
}

// ---- host buffers: copies overlapped with the level-0 kernels --------------
//
// crsolve_solve_host on a classic FP64 plan.  A level-0 chunk of odd blocks
// t0 .. t1-1 reads block rows 2 t0 - 1 .. 2 t1 - 1 of A and B and writes rows
// 2 t0 .. 2 t1 - 1 of x, so level 0 is run as G chunk ranges: on a copy
// stream the rows of A and B are sent range by range (in row order, so the
// one row a range needs from its left neighbour has arrived before it), and
// the factor kernel of range g starts as soon as its rows are on the device;
// y follows while the coarse levels are factored; after the down sweep and
// the coarse up sweeps, x of range g goes back to the host while the next
// range of the level-0 up sweep still runs.  Every kernel does exactly the
// work of crsolve_factor + crsolve_solve, so x is bit-identical to theirs.
constexpr int kHostRanges = 8;
constexpr int kWaveLevels = 3;   // levels 1 .. 3 follow level 0 as a wavefront

cudaEvent_t host_event(crsolve_plan_s *p, size_t i) {
    while (p->xev.size() <= i) {
        cudaEvent_t e;
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
        p->xev.push_back(e);
    }
    return p->xev[i];
}

// Chunk range g of G over n chunks: [n g / G, n (g+1) / G).
int64_t range_edge(int64_t n, int g, int G) { return n * g / G; }

int solve_host_pipelined(crsolve_plan_s *p, int k, const crsolve_z *A_host, const crsolve_z *B_host,
                         const crsolve_z *y_host, crsolve_z *x_host, cudaStream_t s) {
    const int64_t N = p->N;
    const size_t zsz = sizeof(crsolve_z), mm = (size_t)p->m * p->m, mk = (size_t)p->m * k;
    z2 *dA = reinterpret_cast<z2 *>(p->map() + p->offSA), *dB = reinterpret_cast<z2 *>(p->map() + p->offSB);
    z2 *dy = reinterpret_cast<z2 *>(p->map() + p->offSY), *dx = reinterpret_cast<z2 *>(p->map() + p->offSX);
    if (!p->cstream && cudaStreamCreateWithFlags(&p->cstream, cudaStreamNonBlocking) != cudaSuccess) {
        p->cstream = nullptr;
        return CRSOLVE_ECUDA;
    }
    cudaStream_t cs = p->cstream;
    size_t ne = 0;
    // the copy stream starts after everything already queued on s
    cudaEvent_t e = host_event(p, ne++);
    if (!e || cudaEventRecord(e, s) != cudaSuccess || cudaStreamWaitEvent(cs, e, 0) != cudaSuccess)
        return CRSOLVE_ECUDA;
    if (cudaMemsetAsync(p->map() + p->offStatus, 0xFF, sizeof(unsigned long long), s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    int rc;
    // Factor with a wavefront: level 0 by ranges of chunks, each after its
    // rows of A and B; after each range, the chunks of levels 1 ..
    // kWaveLevels whose rows are complete, so the GPU keeps working while the
    // copies run.  A level-l chunk c reads rows 2 c nb .. 2 (c+1) nb - 1 of the
    // level-l system; after chunks 0 .. d-1 of level l and the boundaries
    // between them, rows 0 .. d nb - 2 of level l+1 are complete.  Each wave
    // level writes its CTA-boundary blocks to a region of its own, so chunks
    // of interleaved levels never share one; the later levels run after all
    // of them and reuse the first region.
    const int nlev = (int)p->lev.size();
    struct Wave { crs::LevelArgs a; int64_t nc, done, fixed, rows; };
    std::vector<Wave> w(nlev);
    {
        z2 *wbd = reinterpret_cast<z2 *>(p->map() + p->offWbd);
        const int64_t cap = (N + 1) / 2;   // chunks the boundary region holds
        int64_t used = 0;
        for (int l = 0; l < nlev; ++l) {
            Wave &W = w[l];
            W.a = level_args(p, l, dA, dB);
            W.a.nb = crs::factor_nb(p->mt, W.a.no, p->nsm);
            W.nc = crs::num_ctas(W.a.no, W.a.nb);
            W.done = 0;
            W.fixed = 1;
            W.rows = 0;
            if (l <= kWaveLevels && used + W.nc <= cap) {
                W.a.Wbd = wbd + used * (int64_t)mm;
                used += W.nc;
            } else {
                W.a.Wbd = wbd;
            }
        }
    }
    int wave = 0;   // deepest wave level whose boundary region is its own
    for (int l = 1; l <= kWaveLevels && l < nlev; ++l)
        if (w[l].a.Wbd != w[0].a.Wbd || w[l].nc == 0) wave = l; else break;
    // launch the ready chunks of level l (at least min_new unless all are
    // ready) and the boundaries between done chunks
    auto advance = [&](int l, int64_t min_new) -> int {
        Wave &W = w[l];
        const int64_t ready = W.rows >= W.a.Nl ? W.nc : std::min(W.nc, W.rows / (2 * (int64_t)W.a.nb));
        if (ready < W.nc && ready - W.done < min_new) return CRSOLVE_OK;
        int r;
        if (ready > W.done) {
            W.a.c_begin = W.done;
            W.a.c_count = ready - W.done;
            const int64_t units = std::min(ready * W.a.nb, W.a.no) - W.done * W.a.nb;
            if ((r = launch(p, CRSOLVE_K_FACTOR_ODD, l, units, s, [&] { return crs::launch_factor_odd(p->mt, W.a, s); })))
                return r;
            W.done = ready;
        }
        if (W.done > W.fixed) {
            W.a.c_begin = W.fixed;
            W.a.c_count = W.done - W.fixed;
            if ((r = launch(p, CRSOLVE_K_FACTOR_FIX, l, W.done - W.fixed, s,
                            [&] { return crs::launch_factor_fix(W.a, p->nsm, s); })))
                return r;
            W.fixed = W.done;
        }
        if (l + 1 < nlev) w[l + 1].rows = W.done == W.nc ? w[l + 1].a.Nl : W.done * W.a.nb - 1;
        return CRSOLVE_OK;
    };
    {
        const int64_t nc = w[0].nc, nb0 = w[0].a.nb;
        const int G = (int)(nc < kHostRanges ? nc : kHostRanges);
        for (int g = 0; g < G; ++g) {
            const int64_t c0 = range_edge(nc, g, G), c1 = range_edge(nc, g + 1, G);
            const int64_t r0 = 2 * c0 * nb0, r1 = (g == G - 1) ? N : 2 * c1 * nb0;
            const int64_t b1 = r1 < N - 1 ? r1 : N - 1;
            if (cudaMemcpyAsync(dA + r0 * mm, A_host + r0 * mm, (r1 - r0) * mm * zsz, cudaMemcpyHostToDevice, cs) !=
                cudaSuccess)
                return CRSOLVE_ECUDA;
            if (b1 > r0 && cudaMemcpyAsync(dB + r0 * mm, B_host + r0 * mm, (b1 - r0) * mm * zsz,
                                           cudaMemcpyHostToDevice, cs) != cudaSuccess)
                return CRSOLVE_ECUDA;
            e = host_event(p, ne++);
            if (!e || cudaEventRecord(e, cs) != cudaSuccess || cudaStreamWaitEvent(s, e, 0) != cudaSuccess)
                return CRSOLVE_ECUDA;
            w[0].rows = r1;
            if ((rc = advance(0, 1))) return rc;
            for (int l = 1; l <= wave; ++l)
                if ((rc = advance(l, std::max<int64_t>(1, w[l].nc / kHostRanges)))) return rc;
        }
    }
    // y while the rest is factored
    if (cudaMemcpyAsync(dy, y_host, N * mk * zsz, cudaMemcpyHostToDevice, cs) != cudaSuccess) return CRSOLVE_ECUDA;
    cudaEvent_t ey = host_event(p, ne++);
    if (!ey || cudaEventRecord(ey, cs) != cudaSuccess) return CRSOLVE_ECUDA;
    for (int l = 0; l < nlev; ++l)
        if ((rc = advance(l, 0))) return rc;
    p->factored = true;
    if (cudaStreamWaitEvent(s, ey, 0) != cudaSuccess) return CRSOLVE_ECUDA;
    if ((rc = solve_sweeps(p, k, dy, dx, 1, s))) return rc;
    // level-0 up sweep by ranges, each range's x sent back behind it
    {
        crs::LevelArgs a = solve_args(p, 0, k);
        a.x = dx;
        const int64_t nc = crs::num_ctas(a.no, a.nb);
        const int G = (int)(nc < kHostRanges ? nc : kHostRanges);
        for (int g = 0; g < G; ++g) {
            const int64_t c0 = range_edge(nc, g, G), c1 = range_edge(nc, g + 1, G);
            const int64_t r0 = 2 * c0 * a.nb, r1 = (g == G - 1) ? N : 2 * c1 * a.nb;
            a.c_begin = c0;
            a.c_count = c1 - c0;
            const int64_t units = (c1 * a.nb < a.no ? c1 * a.nb : a.no) - c0 * a.nb;
            if ((rc = launch(p, CRSOLVE_K_SOLVE_UP, 0, units, s, [&] { return crs::launch_solve_up(p->mt, a, s); })))
                return rc;
            e = host_event(p, ne++);
            if (!e || cudaEventRecord(e, s) != cudaSuccess || cudaStreamWaitEvent(cs, e, 0) != cudaSuccess)
                return CRSOLVE_ECUDA;
            if (cudaMemcpyAsync(x_host + r0 * mk, dx + r0 * mk, (r1 - r0) * mk * zsz, cudaMemcpyDeviceToHost, cs) !=
                cudaSuccess)
                return CRSOLVE_ECUDA;
        }
    }
    // s resumes after the last copy
    e = host_event(p, ne++);
    if (!e || cudaEventRecord(e, cs) != cudaSuccess || cudaStreamWaitEvent(s, e, 0) != cudaSuccess)
        return CRSOLVE_ECUDA;
    return CRSOLVE_OK;
}

// ---- mixed precision ------------------------------------------------------

// Factor: FP32 levels 0..lT-1, the level-lT system converted to FP64, FP64
// levels lT.. .  A breakdown in the FP32 levels is re-decided by a full FP64
// factorisation, so that the reported flags are always the FP64 ones.
int mixed_factor(crsolve_plan_s *p, const z2 *A, const z2 *B, cudaStream_t s) {
    const size_t mm = (size_t)p->m * p->m;
    const WsMap ws = p->map();
    p->A64 = reinterpret_cast<const crsolve_z *>(A);
    p->B64 = reinterpret_cast<const crsolve_z *>(B);
    p->fallback = false;
    if (cudaMemsetAsync(ws + p->offStatus, 0xFF, sizeof(unsigned long long), s) != cudaSuccess ||
        cudaMemsetAsync(ws + p->offErr, 0, sizeof(int), s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    int rc;
    if ((rc = launch(p, CRSOLVE_K_CONVERT, 0, p->N, s, [&] {
             return crs::launch_to_f32(A, reinterpret_cast<crs::c2 *>(ws + p->offA32), p->N * (int64_t)mm, p->nsm, s);
         })))
        return rc;
    if (p->N > 1 && (rc = launch(p, CRSOLVE_K_CONVERT, 0, p->N - 1, s, [&] {
                         return crs::launch_to_f32(B, reinterpret_cast<crs::c2 *>(ws + p->offB32),
                                                   (p->N - 1) * (int64_t)mm, p->nsm, s);
                     })))
        return rc;
    for (int l = 0; l < p->lT; ++l) {
        crs::LevelArgsT<float> a = level_args32(p, l);
        a.nb = crs::factor_nb32(p->mt, a.no, p->nsm);
        if ((rc = launch(p, CRSOLVE_K_FACTOR_ODD, l, a.no, s, [&] { return crs::launch_factor_odd(p->mt, a, s); })))
            return rc;
        if (crs::num_ctas(a.no, a.nb) > 1 &&
            (rc = launch(p, CRSOLVE_K_FACTOR_FIX, l, crs::num_ctas(a.no, a.nb) - 1, s,
                         [&] { return crs::launch_factor_fix(a, p->nsm, s); })))
            return rc;
    }
    // the level-lT system to FP64, into the FP64 layout's slot for it
    const LevelPlan &Lb = p->lev32[p->lT - 1];
    if ((rc = launch(p, CRSOLVE_K_CONVERT, p->lT, Lb.ne, s, [&] {
             cudaError_t e = crs::launch_to_f64(reinterpret_cast<const crs::c2 *>(ws + Lb.offAn),
                                                reinterpret_cast<z2 *>(ws + p->lev[p->lT - 1].offAn),
                                                Lb.ne * (int64_t)mm, p->nsm, s);
             if (e != cudaSuccess) return e;
             return crs::launch_to_f64(reinterpret_cast<const crs::c2 *>(ws + Lb.offBn),
                                       reinterpret_cast<z2 *>(ws + p->lev[p->lT - 1].offBn),
                                       (Lb.ne > 1 ? Lb.ne - 1 : 0) * (int64_t)mm, p->nsm, s);
         })))
        return rc;
    for (int l = p->lT; l < (int)p->lev.size(); ++l) {
        crs::LevelArgs a = level_args(p, l, nullptr, nullptr);
        a.nb = crs::factor_nb(p->mt, a.no, p->nsm);
        if ((rc = launch(p, CRSOLVE_K_FACTOR_ODD, l, a.no, s, [&] { return crs::launch_factor_odd(p->mt, a, s); })))
            return rc;
        if (crs::num_ctas(a.no, a.nb) > 1 &&
            (rc = launch(p, CRSOLVE_K_FACTOR_FIX, l, crs::num_ctas(a.no, a.nb) - 1, s,
                         [&] { return crs::launch_factor_fix(a, p->nsm, s); })))
            return rc;
    }
    if (mixed_uses_split(p)) {
        // binary exponents of the rows of [B_{j-1} | A_j | B_j^H] for the residual's splitting
        crs::ResidTcArgs ra{};
        ra.N = p->N; ra.m = p->m; ra.k = 1;
        ra.A = A; ra.B = B;
        ra.erow = reinterpret_cast<int *>(ws + p->offErow);
        ra.dbg = reinterpret_cast<unsigned long long *>(ws + p->offDbg);
        if ((rc = launch(p, CRSOLVE_K_RESIDUAL, 0, p->N, s, [&] { return crs::launch_row_exponents(ra, p->nsm, s); })))
            return rc;
        // the matrix slices of every residual of the refinement, once
        if ((rc = launch(p, CRSOLVE_K_RESIDUAL, 0, p->N, s, [&] {
                 return crs::launch_matrix_image(ra, reinterpret_cast<unsigned char *>(ws + p->offAimg), p->nsm, s);
             })))
            return rc;
    }
    unsigned long long st = 0;
    int err = 0;
    if (cudaMemcpyAsync(&st, ws + p->offStatus, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&err, ws + p->offErr, sizeof(err), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    if (err) return CRSOLVE_ETIMEOUT;
    p->factored = true;
    if (st != CRS_NO_FAIL) {
        p->fallback = true;
        return do_factor(p, A, B, s);
    }
    return CRSOLVE_OK;
}

// One correction solve d = A~^{-1} r with the mixed factorisation: r (FP64)
// -> FP32, FP32 down sweep, FP64 coarse levels, FP32 up sweep -> d (FP32).
int mixed_correction(crsolve_plan_s *p, int k, const z2 *r, cudaStream_t s) {
    const WsMap ws = p->map();
    const int64_t mk = (int64_t)p->m * k;
    const int nlev = (int)p->lev.size();
    int rc;
    if ((rc = launch(p, CRSOLVE_K_CONVERT, 0, p->N, s, [&] {
             return crs::launch_to_f32(r, reinterpret_cast<crs::c2 *>(ws + p->offY32), p->N * mk, p->nsm, s);
         })))
        return rc;
    for (int l = 0; l < p->lT; ++l) {
        crs::LevelArgsT<float> a = level_args32(p, l);
        a.k = k;
        a.nb = crs::solve_nb32(p->mt, a.no, p->nsm);
        a.kc = crs::solve_kc32(p->mt, k, a.no, p->nsm);
        if ((rc = launch(p, CRSOLVE_K_SOLVE_DOWN_ODD, l, a.no, s, [&] { return crs::launch_solve_down_odd(p->mt, a, s); })))
            return rc;
        if (crs::num_ctas(a.no, a.nb) > 1 &&
            (rc = launch(p, CRSOLVE_K_SOLVE_DOWN_FIX, l, crs::num_ctas(a.no, a.nb) - 1, s,
                         [&] { return crs::launch_solve_down_fix(a, p->nsm, s); })))
            return rc;
    }
    const LevelPlan &Lb = p->lev32[p->lT - 1];
    if ((rc = launch(p, CRSOLVE_K_CONVERT, p->lT, Lb.ne, s, [&] {
             return crs::launch_to_f64(reinterpret_cast<const crs::c2 *>(ws + Lb.offYn),
                                       reinterpret_cast<z2 *>(ws + p->lev[p->lT - 1].offYn), Lb.ne * mk, p->nsm, s);
         })))
        return rc;
    for (int l = p->lT; l < nlev; ++l) {
        crs::LevelArgs a = level_args(p, l, nullptr, nullptr);
        a.k = k;
        a.nb = crs::solve_nb(p->mt, a.no, p->nsm);
        a.kc = crs::solve_kc(p->mt, k, a.no, p->nsm);
        a.y = reinterpret_cast<const z2 *>(ws + p->lev[l - 1].offYn);
        if ((rc = launch(p, CRSOLVE_K_SOLVE_DOWN_ODD, l, a.no, s, [&] { return crs::launch_solve_down_odd(p->mt, a, s); })))
            return rc;
        if (crs::num_ctas(a.no, a.nb) > 1 &&
            (rc = launch(p, CRSOLVE_K_SOLVE_DOWN_FIX, l, crs::num_ctas(a.no, a.nb) - 1, s,
                         [&] { return crs::launch_solve_down_fix(a, p->nsm, s); })))
            return rc;
    }
    for (int l = nlev - 1; l >= p->lT; --l) {
        crs::LevelArgs a = level_args(p, l, nullptr, nullptr);
        a.k = k;
        a.nb = crs::solve_nb(p->mt, a.no, p->nsm);
        a.kc = crs::solve_kc(p->mt, k, a.no, p->nsm);
        a.x = reinterpret_cast<z2 *>(ws + p->lev[l - 1].offXn);
        if ((rc = launch(p, CRSOLVE_K_SOLVE_UP, l, a.no, s, [&] { return crs::launch_solve_up(p->mt, a, s); })))
            return rc;
    }
    if ((rc = launch(p, CRSOLVE_K_CONVERT, p->lT, Lb.ne, s, [&] {
             return crs::launch_to_f32(reinterpret_cast<const z2 *>(ws + p->lev[p->lT - 1].offXn),
                                       reinterpret_cast<crs::c2 *>(ws + Lb.offXn), Lb.ne * mk, p->nsm, s);
         })))
        return rc;
    for (int l = p->lT - 1; l >= 0; --l) {
        crs::LevelArgsT<float> a = level_args32(p, l);
        a.k = k;
        a.nb = crs::solve_nb32(p->mt, a.no, p->nsm);
        a.kc = crs::solve_kc32(p->mt, k, a.no, p->nsm);
        if ((rc = launch(p, CRSOLVE_K_SOLVE_UP, l, a.no, s, [&] { return crs::launch_solve_up(p->mt, a, s); })))
            return rc;
    }
    return CRSOLVE_OK;
}

// Mixed-precision solve: preconditioned conjugate gradients (per right-hand-side
// column; A is Hermitian positive definite) with the FP32 cyclic-reduction
// solve A~^{-1} as preconditioner and FP64 matrix-vector products, the
// iterative-refinement scheme of Carson and Higham ("A new analysis of
// iterative refinement and its application to accurate solution of
// ill-conditioned sparse linear systems", SIAM J. Sci. Comput. 39, 2017) with
// CG in place of GMRES.  The preconditioner is applied in FP32 and so is not
// exactly the same linear map from step to step: beta is the flexible
// (Polak-Ribiere) one, (r_{i+1}, z_{i+1} - z_i) / (r_i, z_i).
//
//   x_0 = A~^{-1} y,  r_0 = y - A x_0,  z_0 = p_0 = A~^{-1} r_0
//   w_i = -A p_i,  alpha_i = (r_i, z_i) / (p_i, A p_i)
//   x_{i+1} = x_i + alpha_i p_i,  r_{i+1} = r_i + alpha_i w_i
//   z_{i+1} = A~^{-1} r_{i+1},  p_{i+1} = z_{i+1} + beta_i p_i
//
// The residuals and products are FP64-accurate: for m > 32 (and unless the
// plan asks for the FP64 pipe) by exact splitting on the tensor cores
// (cr_resid_tc.cu), else by FP64 FMA.  Stop rule, with delta_i the largest
// relative correction max_c |alpha p|_c / |x|_c and rho = delta_i /
// delta_{i-1}: stop when delta_i <= kMixedTol, a tenth of the stated bound
// 1e-10 (the error left is about the next correction, smaller still), or when
// the geometric extrapolation rho * delta_i of the remaining error is below
// kMixedTol / 10 with delta_i <= 1e-8 and rho <= 1e-2.  The extrapolation is
// trusted only that late: CG's first steps can shrink the correction by
// orders of magnitude more than the steps after them (measured: 0.055 ->
// 3.3e-7 -> 2.4e-9 at kappa ~ 1e6).  The FP64 path takes over when the
// iteration does not contract (rho > 0.9 twice, rho >= 2, a non-positive
// curvature, NaN) or when the steps still needed at the observed rate would
// cost more than the FP64 factor + solve.
//
// CG updates the residual recursively (r += alpha w); rounding makes it
// drift from the true y - A x by about u * (steps) * |A| |x|, which reaches
// the solution multiplied by kappa.  The first correction estimates kappa
// (delta_1 ~ kappa * u_FP32): above kMixedVerifyAbove (kappa >~ 1e3) the
// first stop is followed by a restart from the true residual (a refinement
// step in the sense of Carson and Higham), and the solve ends at the next
// stop; the drift of the restarted run acts on a residual already reduced by
// the error at the restart.  Measured at kappa ~ 1e6 without the restart:
// corrections down to 1e-16, error 2.8e-9 against the oracle.
constexpr double kMixedTol = 1e-11, kMixedExtrapFrom = 1e-8, kMixedVerifyAbove = 1e-4;

// Cost of one step (an FP32 correction sweep and an FP64-accurate product)
// relative to the FP64 factor + solve, in FP64-pipe flops per block row:
// the FP32 sweep 40 m^2 k flop at about 1/8 of its FP64 time (measured), the
// product 24 m^2 k flop on the FP64 pipe, or about 1/16 of that with the
// tensor-core splitting; the FP64 path 25.33 m^3 + 40 m^2 k.
double mixed_step_cost(int m, int k, bool split) {
    const double mm = (double)m * m, step = (split ? 1.5 : 24.0) * mm * k + 5.0 * mm * k;
    return step / (25.33 * mm * m + 40.0 * mm * k);
}

// r = y - A x (y may be NULL: r = -A x), FP64-accurate.
int mixed_residual(crsolve_plan_s *p, int k, const z2 *x, const z2 *y, z2 *r, cudaStream_t s) {
    const WsMap ws = p->map();
    if (!mixed_uses_split(p)) {
        if (y) {
            return launch(p, CRSOLVE_K_RESIDUAL, 0, p->N, s, [&] {
                return crs::launch_residual(p->N, p->m, k, reinterpret_cast<const z2 *>(p->A64),
                                            reinterpret_cast<const z2 *>(p->B64), x, y, r, p->nsm, s);
            });
        }
        // -A x: the FP64 kernel subtracts from a zero right-hand side
        if (cudaMemsetAsync(r, 0, p->N * (size_t)p->m * k * sizeof(z2), s) != cudaSuccess) return CRSOLVE_ECUDA;
        return launch(p, CRSOLVE_K_RESIDUAL, 0, p->N, s, [&] {
            return crs::launch_residual(p->N, p->m, k, reinterpret_cast<const z2 *>(p->A64),
                                        reinterpret_cast<const z2 *>(p->B64), x, r, r, p->nsm, s);
        });
    }
    crs::ResidTcArgs a{};
    a.N = p->N; a.m = p->m; a.k = k;
    a.A = reinterpret_cast<const z2 *>(p->A64);
    a.B = reinterpret_cast<const z2 *>(p->B64);
    a.x = x; a.y = y; a.r = r;
    a.erow = reinterpret_cast<int *>(ws + p->offErow);
    a.ecol = reinterpret_cast<int *>(ws + p->offEcol);
    a.err = reinterpret_cast<int *>(ws + p->offErr);
    a.dbg = reinterpret_cast<unsigned long long *>(ws + p->offDbg);
    a.img = reinterpret_cast<const unsigned char *>(ws + p->offAimg);
    return launch(p, CRSOLVE_K_RESIDUAL, 0, p->N, s, [&] { return crs::launch_residual_tc(a, p->nsm, s); });
}

int mixed_solve(crsolve_plan_s *p, int k, const z2 *y, z2 *x, cudaStream_t s) {
    const WsMap ws = p->map();
    const int64_t rows = p->N * (int64_t)p->m, n = rows * k;
    unsigned long long *norms = reinterpret_cast<unsigned long long *>(ws + p->offNorms);
    z2 *r = reinterpret_cast<z2 *>(ws + p->offR64);
    z2 *pd = reinterpret_cast<z2 *>(ws + p->offP64);
    z2 *w = reinterpret_cast<z2 *>(ws + p->offW64);
    const crs::c2 *z = reinterpret_cast<const crs::c2 *>(ws + p->offX32);
    double *part = reinterpret_cast<double *>(ws + p->offDot);
    double *alpha = reinterpret_cast<double *>(ws + p->offScal);
    double *beta = alpha + p->kmax, *rz = beta + p->kmax, *rzc = rz + p->kmax;
    int *errw = reinterpret_cast<int *>(ws + p->offErr);   // [0] a bounded wait gave up, [1] curvature lost
    int *flag = errw + 1;
    int rc;
    const size_t kb = (size_t)k * sizeof(unsigned long long);
    p->last_iters = 0;
    p->last_delta = p->last_rho = 0.0;
    if (cudaMemsetAsync(flag, 0, sizeof(int), s) != cudaSuccess) return CRSOLVE_ECUDA;
    // x_0 = A~^{-1} y
    if ((rc = mixed_correction(p, k, y, s))) return rc;
    if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s,
                     [&] { return crs::launch_update(x, z, n, 1, norms, p->nsm, s); })))
        return rc;
    // r_0 = y - A x_0, z_0 = A~^{-1} r_0, p_0 = z_0, rz = (r_0, z_0)
    if ((rc = mixed_residual(p, k, x, y, r, s))) return rc;
    p->last_iters = 1;
    if ((rc = mixed_correction(p, k, r, s))) return rc;
    if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s,
                     [&] { return crs::launch_pcg_direction(pd, z, beta, n, k, 1, p->nsm, s); })))
        return rc;
    if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s, [&] {
             return crs::launch_dot(r, z, rows, k, part, rz, 0, nullptr, nullptr, nullptr, p->nsm, s);
         })))
        return rc;
    double prev = 0.0;
    int slow = 0, since = 0;
    bool verify = false, restarted = false;
    std::vector<unsigned long long> hn(2 * (size_t)k);
    for (int it = 1; it <= kMixedMaxIter; ++it) {
        ++since;
        // w = -A p, alpha = (r, z) / (p, A p)
        if ((rc = mixed_residual(p, k, pd, nullptr, w, s))) return rc;
        p->last_iters += 1;
        if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s, [&] {
                 return crs::launch_dot(pd, w, rows, k, part, alpha, 1, rz, nullptr, flag, p->nsm, s);
             })))
            return rc;
        // x += alpha p, r += alpha w, and the column maxima of the correction and of x
        if (cudaMemsetAsync(norms, 0, 2 * kb, s) != cudaSuccess) return CRSOLVE_ECUDA;
        if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s, [&] {
                 return crs::launch_pcg_update(x, r, pd, w, alpha, n, k, norms, p->nsm, s);
             })))
            return rc;
        int hflag[2] = {0, 0};
        if (cudaMemcpyAsync(hn.data(), norms, 2 * kb, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaMemcpyAsync(hflag, errw, sizeof(hflag), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess)
            return CRSOLVE_ECUDA;
        if (hflag[0]) return CRSOLVE_ETIMEOUT;
        double delta = 0.0;
        for (int c = 0; c < k; ++c) {
            double dn, xn;
            memcpy(&dn, &hn[c], 8);
            memcpy(&xn, &hn[k + c], 8);
            const double dc = xn > 0 ? dn / xn : (dn > 0 ? 1.0 : 0.0);
            delta = (dc == dc && delta == delta) ? std::max(delta, dc) : NAN;
        }
        if (hflag[1] || !(delta == delta)) break;           // lost positive curvature or NaN: FP64
        const double rho = since > 1 ? (prev > 0 ? delta / prev : 0.0) : 0.0;
        p->last_delta = delta;
        p->last_rho = rho;
        if (it == 1) verify = delta > kMixedVerifyAbove;
        // the correction itself below the tolerance, or (extrapolation) a fast,
        // small contraction that puts the remaining error a decade below it
        const bool extrap = since > 1 && delta <= kMixedExtrapFrom && rho <= 1e-2 && rho * delta <= 0.1 * kMixedTol;
        if (delta <= kMixedTol || extrap) {
            if (!verify || restarted) return CRSOLVE_OK;
            // the recursive residual may have drifted from y - A x: restart
            // from the true residual (one refinement step) and go on
            restarted = true;
            since = 0;
            prev = 0.0;
            slow = 0;
            if ((rc = mixed_residual(p, k, x, y, r, s))) return rc;
            p->last_iters += 1;
            if ((rc = mixed_correction(p, k, r, s))) return rc;
            if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s,
                             [&] { return crs::launch_pcg_direction(pd, z, beta, n, k, 1, p->nsm, s); })))
                return rc;
            if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s, [&] {
                     return crs::launch_dot(r, z, rows, k, part, rz, 0, nullptr, nullptr, nullptr, p->nsm, s);
                 })))
                return rc;
            continue;
        }
        if (since > 1) {
            slow = rho > 0.9 ? slow + 1 : 0;
            if (slow >= 2 || !(rho < 2.0)) break;
            if (rho < 1.0) {
                // steps still needed for rho^n * delta <= kMixedTol, against the FP64 path
                const double need = std::ceil(std::log(kMixedTol / (rho * delta)) / std::log(rho));
                if (need * mixed_step_cost(p->m, k, mixed_uses_split(p)) > 1.0) break;
            }
        }
        prev = delta;
        // beta = (r_{i+1}, z_{i+1} - z_i) / (r_i, z_i): (r_{i+1}, z_i) first, while z still holds z_i
        if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s, [&] {
                 return crs::launch_dot(r, z, rows, k, part, rzc, 0, nullptr, nullptr, nullptr, p->nsm, s);
             })))
            return rc;
        if ((rc = mixed_correction(p, k, r, s))) return rc;
        if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s, [&] {
                 return crs::launch_dot(r, z, rows, k, part, beta, 2, rz, rzc, nullptr, p->nsm, s);
             })))
            return rc;
        if ((rc = launch(p, CRSOLVE_K_UPDATE, 0, p->N, s,
                         [&] { return crs::launch_pcg_direction(pd, z, beta, n, k, 0, p->nsm, s); })))
            return rc;
    }
    // no convergence in mixed precision: factor and solve in FP64
    p->fallback = true;
    if ((rc = do_factor(p, reinterpret_cast<const z2 *>(p->A64), reinterpret_cast<const z2 *>(p->B64), s))) return rc;
    return do_solve(p, k, y, x, s);
}

// Workspace layout of a plan (offsets; see WsMap for the two regions).
void layout(crsolve_plan_s *p) {
    const int64_t N = p->N;
    const int m = p->m;
    const bool alg1 = p->alg1;
    const uint32_t flags = p->flags;
    const int precision = p->precision;
    const size_t zsz = sizeof(crsolve_z), mm = (size_t)m * m, mk = (size_t)m * p->kmax;
    size_t cur = 0, scur = 0;
    // region of the keep_levels split: tp = workspace, ts = scratch (the
    // workspace too when the plan is not split)
    const bool split = p->keep >= 0;
    auto tp = [&](size_t bytes) { return take(cur, bytes); };
    auto ts = [&](size_t bytes) { return split ? (take(scur, bytes) | kScr) : take(cur, bytes); };
    p->lev.clear();
    p->lev32.clear();
    p->alev[0].clear();
    p->alev[1].clear();
    p->offStatus = take(cur, 256);
    p->offDbg = take(cur, 256);
    if (alg1) {
        int L = 0;
        while ((int64_t(1) << L) < N) ++L;
        p->aL = L;
        for (int l = 0; l <= L; ++l)
            for (int h = 0; h < 2; ++h) {
                if (h == 1 && N < 2) continue;
                LevelPlan H{};
                H.Nl = N + h; H.no = (H.Nl + 1) / 2; H.ne = H.Nl / 2;
                H.offL = take(cur, H.no * mm * zsz);
                H.offInv = take(cur, H.no * (size_t)m * sizeof(double));
                H.offZ = take(cur, H.no * 2 * mm * zsz);
                p->alev[h].push_back(H);
            }
        const int64_t noB = N / 2 + 1;
        for (int b = 0; b < 2; ++b) {
            p->offA1A[b] = take(cur, (N + 1) * mm * zsz);
            p->offA1B[b] = take(cur, N * mm * zsz);
            p->offA1Y[b] = take(cur, (N + 1) * mk * zsz);
        }
        p->offA1R[0] = take(cur, ((N + 1) / 2) * mk * zsz);
        p->offA1R[1] = take(cur, noB * mk * zsz);
        p->offA1Xb = take(cur, (N + 1) * mk * zsz);
        p->offA1Xz = take(cur, noB * mk * zsz);
        p->offWbd = take(cur, noB * mm * zsz);
        p->offCbd = take(cur, noB * mk * zsz);
    }
    int64_t Nl = N;
    while (!alg1) {
        LevelPlan L{};
        L.Nl = Nl; L.no = (Nl + 1) / 2; L.ne = Nl / 2;
        // factors of levels < keep (and the level-keep system) persist
        const bool keep_l = !split || (int)p->lev.size() < p->keep;
        auto tf = [&](size_t bytes) { return keep_l ? tp(bytes) : ts(bytes); };
        L.offL = tf(L.no * mm * zsz);
        L.offInv = tf(L.no * (size_t)m * sizeof(double));
        L.offZ = tf(L.no * 2 * mm * zsz);
        L.offR = ts(L.no * mk * zsz);
        L.offAn = tf(L.ne * mm * zsz);
        L.offBn = tf((L.ne > 1 ? L.ne - 1 : 0) * mm * zsz);
        L.offYn = ts(L.ne * mk * zsz);
        L.offXn = ts(L.ne * mk * zsz);
        p->lev.push_back(L);
        if (Nl == 1) break;
        Nl /= 2;
    }
    const int64_t no0 = (N + 1) / 2;
    // CTA-boundary scratch: at most one m x m (factor) and one m x kmax (solve)
    // per CTA of the largest level
    if (!alg1) {
        p->offWbd = ts(no0 * mm * zsz);
        p->offCbd = ts(no0 * mk * zsz);
        p->bdc_cap = no0 * (int64_t)p->kmax;
        p->offBdc = ts((size_t)p->bdc_cap * sizeof(unsigned));
    }
    if (flags & CRSOLVE_PLAN_HOST_STAGING) {
        p->offSA = ts(N * mm * zsz);
        p->offSB = ts((N - 1) * mm * zsz);
        p->offSY = ts(N * mk * zsz);
        p->offSX = ts(N * mk * zsz);
    }
    if (precision == CRSOLVE_MIXED) {
        // FP32 levels: all levels with more than kMixedCoarse blocks (at least one)
        int lT = 0;
        while (lT + 1 < (int)p->lev.size() && p->lev[lT].Nl > kMixedCoarse) ++lT;
        if (lT == 0) lT = p->lev.size() > 1 ? 1 : 0;
        p->lT = lT;
        const size_t c32 = 8;
        for (int l = 0; l < lT; ++l) {
            const LevelPlan &L64 = p->lev[l];
            LevelPlan L{};
            L.Nl = L64.Nl; L.no = L64.no; L.ne = L64.ne;
            L.offL = take(cur, L.no * mm * c32);
            L.offInv = take(cur, L.no * (size_t)m * 4);
            L.offZ = take(cur, L.no * 2 * mm * c32);
            L.offR = take(cur, L.no * mk * c32);
            L.offAn = take(cur, L.ne * mm * c32);
            L.offBn = take(cur, (L.ne > 1 ? L.ne - 1 : 0) * mm * c32);
            L.offYn = take(cur, L.ne * mk * c32);
            L.offXn = take(cur, L.ne * mk * c32);
            p->lev32.push_back(L);
        }
        p->offWbd32 = take(cur, no0 * mm * c32);
        p->offCbd32 = take(cur, no0 * mk * c32);
        p->offA32 = take(cur, N * mm * c32);
        p->offB32 = take(cur, (N - 1) * mm * c32);
        p->offY32 = take(cur, N * mk * c32);
        p->offX32 = take(cur, N * mk * c32);
        p->offR64 = take(cur, N * mk * zsz);
        p->offNorms = take(cur, 2 * (size_t)p->kmax * sizeof(unsigned long long));
        p->offErr = take(cur, 16);
        p->offP64 = take(cur, N * mk * zsz);
        p->offW64 = take(cur, N * mk * zsz);
        p->offDot = take(cur, (size_t)crs::dot_partials(p->nsm) * p->kmax * sizeof(double));
        p->offScal = take(cur, 5 * (size_t)p->kmax * sizeof(double));
        p->offErow = take(cur, (size_t)N * m * sizeof(int));
        p->offEcol = take(cur, (size_t)N * p->kmax * sizeof(int));
        if (mixed_uses_split(p)) p->offAimg = take(cur, crs::residual_image_bytes(N));
    }
    p->total = cur;
    p->scr_total = scur;
}

}  // namespace

extern "C" {

int crsolve_plan_create(int64_t N, int32_t m, int32_t kmax, int32_t precision, uint32_t flags,
                        crsolve_plan *out_plan) {
    if (!out_plan) return CRSOLVE_EINVAL;
    *out_plan = nullptr;
    if (N < 1 || m < 1 || kmax < 1) return CRSOLVE_EINVAL;
    if (m > CRSOLVE_MAX_M || kmax > CRSOLVE_MAX_K) return CRSOLVE_EUNSUPPORTED;
    if (precision != CRSOLVE_FP64 && precision != CRSOLVE_MIXED) return CRSOLVE_EUNSUPPORTED;
    if (flags & ~(uint32_t)(CRSOLVE_PLAN_HOST_STAGING | CRSOLVE_PLAN_ALG1 | CRSOLVE_PLAN_FP64_RESIDUAL))
        return CRSOLVE_EINVAL;
    const bool alg1 = (flags & CRSOLVE_PLAN_ALG1) != 0;
    if (alg1 && ((N & (N - 1)) != 0 || precision != CRSOLVE_FP64)) return CRSOLVE_EUNSUPPORTED;
    crsolve_plan_s *p = new (std::nothrow) crsolve_plan_s();
    if (!p) return CRSOLVE_ENOMEM;
    p->N = N; p->m = m; p->kmax = kmax; p->precision = precision; p->flags = flags;
    p->mt = crs::pick_mt(m);
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        delete p;
        return CRSOLVE_ECUDA;
    }
    p->alg1 = alg1;
    layout(p);
    *out_plan = p;
    return CRSOLVE_OK;
}

int crsolve_plan_keep_levels(crsolve_plan p, int32_t keep) {
    if (!p || keep < -1 || p->ws || p->scr) return CRSOLVE_EINVAL;
    if (keep >= 0 && (p->alg1 || p->precision != CRSOLVE_FP64)) return CRSOLVE_EUNSUPPORTED;
    p->keep = keep;
    layout(p);
    p->factored = false;
    p->coarse_valid = false;
    return CRSOLVE_OK;
}

int crsolve_scratch_bytes(crsolve_plan p, size_t *bytes) {
    if (!p || !bytes) return CRSOLVE_EINVAL;
    *bytes = p->scr_total;
    return CRSOLVE_OK;
}

int crsolve_set_scratch(crsolve_plan p, void *dev_ptr, size_t bytes) {
    if (!p || p->keep < 0) return CRSOLVE_EINVAL;
    if (dev_ptr && ((uintptr_t)dev_ptr & 255u)) return CRSOLVE_EINVAL;
    if (dev_ptr && bytes < p->scr_total) return CRSOLVE_ENOMEM;
    p->scr = static_cast<char *>(dev_ptr);
    p->coarse_valid = false;
    return CRSOLVE_OK;
}

int crsolve_workspace_bytes(crsolve_plan p, size_t *bytes) {
    if (!p || !bytes) return CRSOLVE_EINVAL;
    *bytes = p->total;
    return CRSOLVE_OK;
}

int crsolve_set_workspace(crsolve_plan p, void *dev_ptr, size_t bytes) {
    if (!p || !dev_ptr || ((uintptr_t)dev_ptr & 255u)) return CRSOLVE_EINVAL;
    if (bytes < p->total) return CRSOLVE_ENOMEM;
    p->ws = static_cast<char *>(dev_ptr);
    p->ws_bytes = bytes;
    p->factored = false;
    return CRSOLVE_OK;
}

int crsolve_factor(crsolve_plan p, const crsolve_z *A, const crsolve_z *B, void *stream) {
    NvtxRange nv("crsolve_factor");
    if (!p || !A || (p->N > 1 && !B)) return CRSOLVE_EINVAL;
    if (!aligned16(A) || (B && !aligned16(B))) return CRSOLVE_EINVAL;
    if (!p->ws || (p->keep >= 0 && !p->scr)) return CRSOLVE_ENOMEM;
    int rc = check_device(p);
    if (rc) return rc;
    if ((rc = ensure_prepared(p))) return rc;
    if ((rc = debug_reset(p, static_cast<cudaStream_t>(stream)))) return rc;
    if (p->precision == CRSOLVE_MIXED && p->lT > 0)
        return mixed_factor(p, reinterpret_cast<const z2 *>(A), reinterpret_cast<const z2 *>(B),
                            static_cast<cudaStream_t>(stream));
    p->coarse_valid = false;
    if ((rc = do_factor(p, reinterpret_cast<const z2 *>(A), reinterpret_cast<const z2 *>(B),
                        static_cast<cudaStream_t>(stream))))
        return rc;
    p->coarse_valid = true;
    p->lvl0A = reinterpret_cast<const z2 *>(A);
    p->lvl0B = reinterpret_cast<const z2 *>(B);
    return CRSOLVE_OK;
}

int crsolve_solve(crsolve_plan p, int32_t k, const crsolve_z *y, crsolve_z *x, void *stream) {
    NvtxRange nv("crsolve_solve");
    if (!p || !y || !x || k < 1) return CRSOLVE_EINVAL;
    if (k > p->kmax) return CRSOLVE_EUNSUPPORTED;
    if (!aligned16(y) || !aligned16(x) || (const void *)y == (const void *)x) return CRSOLVE_EINVAL;
    if (!p->ws || (p->keep >= 0 && !p->scr)) return CRSOLVE_ENOMEM;
    if (!p->factored) return CRSOLVE_ENOTFACTORED;
    int rc = check_device(p);
    if (rc) return rc;
    if ((rc = ensure_prepared(p))) return rc;
    if (p->precision == CRSOLVE_MIXED && p->lT > 0 && !p->fallback)
        return mixed_solve(p, k, reinterpret_cast<const z2 *>(y), reinterpret_cast<z2 *>(x),
                           static_cast<cudaStream_t>(stream));
    if ((rc = ensure_coarse(p, static_cast<cudaStream_t>(stream)))) return rc;
    return do_solve(p, k, reinterpret_cast<const z2 *>(y), reinterpret_cast<z2 *>(x),
                    static_cast<cudaStream_t>(stream));
}

int crsolve_mixed_precondition(crsolve_plan p, int32_t k, const crsolve_z *r, crsolve_z *z, void *stream) {
    NvtxRange nv("crsolve_mixed_precondition");
    if (!p || !r || !z || k < 1) return CRSOLVE_EINVAL;
    if (k > p->kmax) return CRSOLVE_EUNSUPPORTED;
    if (!aligned16(r) || !aligned16(z)) return CRSOLVE_EINVAL;
    if (!p->ws || (p->keep >= 0 && !p->scr)) return CRSOLVE_ENOMEM;
    if (!p->factored) return CRSOLVE_ENOTFACTORED;
    if (p->precision != CRSOLVE_MIXED || p->lT == 0 || p->fallback) return CRSOLVE_EUNSUPPORTED;
    int rc = check_device(p);
    if (rc) return rc;
    if ((rc = ensure_prepared(p))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // r is read (into the FP32 right-hand side) before z is written, so they may alias
    if ((rc = mixed_correction(p, k, reinterpret_cast<const z2 *>(r), s))) return rc;
    const crs::c2 *z32 = reinterpret_cast<const crs::c2 *>(p->map() + p->offX32);
    return launch(p, CRSOLVE_K_CONVERT, 0, p->N, s, [&] {
        return crs::launch_to_f64(z32, reinterpret_cast<z2 *>(z), p->N * (int64_t)p->m * k, p->nsm, s);
    });
}

int crsolve_backward(crsolve_plan p, int32_t k, const crsolve_z *x, const crsolve_z *gx, crsolve_z *gy,
                     crsolve_z *gA, crsolve_z *gB, void *stream) {
    NvtxRange nv("crsolve_backward");
    if (!p || !x || !gx || !gy || k < 1) return CRSOLVE_EINVAL;
    if (k > p->kmax) return CRSOLVE_EUNSUPPORTED;
    if (!aligned16(x) || !aligned16(gx) || !aligned16(gy) || (gA && !aligned16(gA)) ||
        (gB && !aligned16(gB)))
        return CRSOLVE_EINVAL;
    if ((const void *)gx == (const void *)gy) return CRSOLVE_EINVAL;
    if (p->N == 1) gB = nullptr;
    if (!p->ws || (p->keep >= 0 && !p->scr)) return CRSOLVE_ENOMEM;
    if (!p->factored) return CRSOLVE_ENOTFACTORED;
    int rc = check_device(p);
    if (rc) return rc;
    if ((rc = ensure_prepared(p))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = ensure_coarse(p, s))) return rc;
    if ((rc = do_solve(p, k, reinterpret_cast<const z2 *>(gx), reinterpret_cast<z2 *>(gy), s))) return rc;
    if (!gA && !gB) return CRSOLVE_OK;
    if ((rc = launch(p, CRSOLVE_K_ADJOINT, 0, p->N, s, [&] {
             return crs::launch_adjoint_outer(p->N, p->m, k, reinterpret_cast<const z2 *>(x),
                                              reinterpret_cast<const z2 *>(gy), reinterpret_cast<z2 *>(gA),
                                              reinterpret_cast<z2 *>(gB), p->nsm, s);
         })))
        return rc;
    const unsigned long long *st = reinterpret_cast<const unsigned long long *>(p->map() + p->offStatus);
    const int64_t mm = (int64_t)p->m * p->m;
    if (gA && (rc = launch(p, CRSOLVE_K_NANFILL, 0, p->N, s, [&] {
                   return crs::launch_nan_if_failed(reinterpret_cast<z2 *>(gA), p->N * mm, st, p->nsm, s);
               })))
        return rc;
    if (gB && (rc = launch(p, CRSOLVE_K_NANFILL, 0, p->N - 1, s, [&] {
                   return crs::launch_nan_if_failed(reinterpret_cast<z2 *>(gB), (p->N - 1) * mm, st, p->nsm, s);
               })))
        return rc;
    return CRSOLVE_OK;
}

int crsolve_solve_host(crsolve_plan p, int32_t k, const crsolve_z *A_host, const crsolve_z *B_host,
                       const crsolve_z *y_host, crsolve_z *x_host, void *stream) {
    NvtxRange nv("crsolve_solve_host");
    if (!p || !A_host || !y_host || !x_host || (p->N > 1 && !B_host) || k < 1) return CRSOLVE_EINVAL;
    if (!(p->flags & CRSOLVE_PLAN_HOST_STAGING)) return CRSOLVE_EINVAL;
    if (k > p->kmax) return CRSOLVE_EUNSUPPORTED;
    if (!p->ws || (p->keep >= 0 && !p->scr)) return CRSOLVE_ENOMEM;
    int rc = check_device(p);
    if (rc) return rc;
    if ((rc = ensure_prepared(p))) return rc;
    if ((rc = debug_reset(p, static_cast<cudaStream_t>(stream)))) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the level-0 system is staged in the scratch region: a split plan can
    // rebuild its coarse levels from level keep >= 1 later, not from level 0
    p->coarse_valid = true;
    p->lvl0A = p->lvl0B = nullptr;
    // the host path factors in FP64: later crsolve_solve calls on a mixed
    // plan must use these factors, not FP32 ones from an earlier crsolve_factor
    if (p->precision == CRSOLVE_MIXED) p->fallback = true;
    const size_t zsz = sizeof(crsolve_z), mm = (size_t)p->m * p->m, mk = (size_t)p->m * k;
    z2 *dA = reinterpret_cast<z2 *>(p->map() + p->offSA), *dB = reinterpret_cast<z2 *>(p->map() + p->offSB);
    z2 *dy = reinterpret_cast<z2 *>(p->map() + p->offSY), *dx = reinterpret_cast<z2 *>(p->map() + p->offSX);
    if (!p->alg1 && p->N > 1) {
        if ((rc = solve_host_pipelined(p, k, A_host, B_host, y_host, x_host, s))) return rc;
    } else {
        if (cudaMemcpyAsync(dA, A_host, p->N * mm * zsz, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return CRSOLVE_ECUDA;
        if (p->N > 1 && cudaMemcpyAsync(dB, B_host, (p->N - 1) * mm * zsz, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return CRSOLVE_ECUDA;
        if (cudaMemcpyAsync(dy, y_host, p->N * mk * zsz, cudaMemcpyHostToDevice, s) != cudaSuccess)
            return CRSOLVE_ECUDA;
        if ((rc = do_factor(p, dA, p->N > 1 ? dB : nullptr, s))) return rc;
        if ((rc = do_solve(p, k, dy, dx, s))) return rc;
        if (cudaMemcpyAsync(x_host, dx, p->N * mk * zsz, cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return CRSOLVE_ECUDA;
    }
    unsigned long long st = 0;
    if (cudaMemcpyAsync(&st, p->map() + p->offStatus, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CRSOLVE_ECUDA;
    return st == CRS_NO_FAIL ? CRSOLVE_OK : CRSOLVE_NOT_PD;
}

int crsolve_info_get(crsolve_plan p, crsolve_info *out, void *stream) {
    if (!p || !out) return CRSOLVE_EINVAL;
    if (!p->ws) return CRSOLVE_ENOMEM;
    if (!p->factored) return CRSOLVE_ENOTFACTORED;
    unsigned long long st = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&st, p->map() + p->offStatus, sizeof(st), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return CRSOLVE_ECUDA;
    if (st == CRS_NO_FAIL) {
        *out = crsolve_info{CRSOLVE_OK, 0, 0, 0};
    } else {
        const int level = (int)(st >> 40);
        const int64_t idx = (int64_t)(st & ((1ull << 40) - 1));
        if (p->alg1) {
            // the kernels report the original block; its position at that
            // level is rotr^level on log2 N bits
            const int L = p->aL, sh = L ? level % L : 0;
            const uint64_t mask = L ? ((1ull << L) - 1) : 0, u = (uint64_t)(idx - 1) & mask;
            const uint64_t pos = sh ? (((u >> sh) | (u << (L - sh))) & mask) : u;
            *out = crsolve_info{CRSOLVE_NOT_PD, level, (int64_t)pos + 1, idx};
        } else {
            *out = crsolve_info{CRSOLVE_NOT_PD, level, idx, idx << level};
        }
    }
    return CRSOLVE_OK;
}

int crsolve_destroy(crsolve_plan p) {
    if (!p) return CRSOLVE_EINVAL;
    for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
    for (cudaEvent_t e : p->xev) cudaEventDestroy(e);
    if (p->cstream) cudaStreamDestroy(p->cstream);
    delete p;
    return CRSOLVE_OK;
}

int crsolve_timing_enable(crsolve_plan p, int32_t enable) {
    if (!p) return CRSOLVE_EINVAL;
    p->timing = enable != 0;
    p->recs.clear();
    p->pool_used = 0;
    return CRSOLVE_OK;
}

int crsolve_timing_read(crsolve_plan p, crsolve_kernel_time *out, int32_t cap, int32_t *count) {
    if (!p || !count || (cap > 0 && !out)) return CRSOLVE_EINVAL;
    *count = (int32_t)p->recs.size();
    for (size_t i = 0; i < p->recs.size(); ++i) {
        const auto &r = p->recs[i];
        if (cudaEventSynchronize(r.e1) != cudaSuccess) return CRSOLVE_ECUDA;
        if ((int32_t)i < cap) {
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, r.e0, r.e1) != cudaSuccess) return CRSOLVE_ECUDA;
            out[i] = crsolve_kernel_time{r.kind, r.level, r.units, ms};
        }
    }
    p->recs.clear();
    p->pool_used = 0;
    return CRSOLVE_OK;
}

int crsolve_mixed_stats(crsolve_plan p, int32_t *iterations, double *delta, double *rho, int32_t *fp64_fallback) {
    if (!p) return CRSOLVE_EINVAL;
    if (iterations) *iterations = p->last_iters;
    if (delta) *delta = p->last_delta;
    if (rho) *rho = p->last_rho;
    if (fp64_fallback) *fp64_fallback = p->fallback ? 1 : 0;
    return CRSOLVE_OK;
}

int crsolve_launch_count(crsolve_plan p, int64_t *count) {
    if (!p || !count) return CRSOLVE_EINVAL;
    *count = p->launches;
    return CRSOLVE_OK;
}

const char *crsolve_strerror(int code) {
    switch (code) {
        case CRSOLVE_OK: return "ok";
        case CRSOLVE_NOT_PD: return "matrix is not positive definite (Cholesky breakdown)";
        case CRSOLVE_EINVAL: return "invalid argument";
        case CRSOLVE_ENOMEM: return "workspace missing or too small";
        case CRSOLVE_ECUDA: return "CUDA runtime error";
        case CRSOLVE_ETIMEOUT: return "device-side wait timed out";
        case CRSOLVE_ENOTFACTORED: return "plan has not been factored";
        case CRSOLVE_EUNSUPPORTED: return "unsupported size or precision";
        default: return "unknown status";
    }
}

int crsolve_tile_set(int32_t mt, int32_t nb_factor, int32_t nb_solve, int32_t kc, int32_t threads,
                     int32_t threads_solve) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return CRSOLVE_ECUDA;
    return crs::set_tile_shape(mt, crs::TileShape{nb_factor, nb_solve, kc, threads, threads_solve}, (size_t)optin)
               ? CRSOLVE_OK
               : CRSOLVE_EINVAL;
}

int crsolve_tile_set_mixed(int32_t mt, int32_t nb_factor, int32_t nb_solve, int32_t kc, int32_t threads,
                           int32_t threads_solve) {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return CRSOLVE_ECUDA;
    return crs::set_tile_shape32(mt, crs::TileShape{nb_factor, nb_solve, kc, threads, threads_solve}, (size_t)optin)
               ? CRSOLVE_OK
               : CRSOLVE_EINVAL;
}

int crsolve_tile_get_mixed(int32_t mt, int32_t *nb_factor, int32_t *nb_solve, int32_t *kc, int32_t *threads,
                           int32_t *threads_solve) {
    if (!nb_factor || !nb_solve || !kc || !threads || !threads_solve) return CRSOLVE_EINVAL;
    const crs::TileShape ts = crs::tile_shape32(mt);
    if (ts.threads == 0) return CRSOLVE_EINVAL;
    *nb_factor = ts.nb_factor; *nb_solve = ts.nb_solve; *kc = ts.kc_max; *threads = ts.threads;
    *threads_solve = ts.threads_solve;
    return CRSOLVE_OK;
}

int crsolve_tile_get(int32_t mt, int32_t *nb_factor, int32_t *nb_solve, int32_t *kc, int32_t *threads,
                     int32_t *threads_solve) {
    if (!nb_factor || !nb_solve || !kc || !threads || !threads_solve) return CRSOLVE_EINVAL;
    const crs::TileShape ts = crs::tile_shape(mt);
    if (ts.threads == 0) return CRSOLVE_EINVAL;
    *nb_factor = ts.nb_factor; *nb_solve = ts.nb_solve; *kc = ts.kc_max; *threads = ts.threads;
    *threads_solve = ts.threads_solve;
    return CRSOLVE_OK;
}

int crsolve_debug_bounds(crsolve_plan p, uint64_t *record, void *stream) {
    if (!p || !record) return CRSOLVE_EINVAL;
#ifdef CRSOLVE_DEBUG_BOUNDS
    if (!p->ws) return CRSOLVE_ENOMEM;
    unsigned long long v = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&v, p->ws + p->offDbg, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    *record = v;
    return CRSOLVE_OK;
#else
    (void)stream;
    *record = ~0ull;
    return CRSOLVE_EUNSUPPORTED;
#endif
}

int crsolve_plan_levels(crsolve_plan p, int32_t *nlev, int64_t *sizes) {
    if (!p || !nlev) return CRSOLVE_EINVAL;
    if (p->alg1) {
        // every level of Algorithm 1 holds all N blocks (2^l systems of N/2^l)
        *nlev = p->aL + 1;
        if (sizes)
            for (int l = 0; l <= p->aL; ++l) sizes[l] = p->N;
        return CRSOLVE_OK;
    }
    *nlev = (int32_t)p->lev.size();
    if (sizes)
        for (size_t l = 0; l < p->lev.size(); ++l) sizes[l] = p->lev[l].Nl;
    return CRSOLVE_OK;
}

int crsolve_debug_level_system(crsolve_plan p, int32_t level, const crsolve_z **A_l, const crsolve_z **B_l) {
    if (!p || !A_l || !B_l || level < 1 || level >= (int32_t)p->lev.size()) return CRSOLVE_EINVAL;
    if (!p->ws) return CRSOLVE_ENOMEM;
    *A_l = reinterpret_cast<const crsolve_z *>(p->map() + p->lev[level - 1].offAn);
    *B_l = reinterpret_cast<const crsolve_z *>(p->map() + p->lev[level - 1].offBn);
    return CRSOLVE_OK;
}

}  // extern "C"
