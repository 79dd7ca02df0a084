// cr_batched.cu -- many independent systems of uneven N, m, k in one
// persistent launch (the paper notes that the block formulas of a level are
// independent across blocks, Sec. 2; independent systems are independent a
// fortiori).
//
// Design.  The grid is one persistent CTA per workspace slot.  A CTA takes the
// next system from an atomic counter (systems ordered by decreasing cost, the
// longest-processing-time-first rule, so that the big systems do not start
// last) and runs the whole classic cyclic reduction of that system: for every
// level the factor chunks and the down-sweep chunks, then the up sweep, with
// the same per-chunk device functions as the level kernels (cr_core.cuh).
// Because one CTA runs the chunks of a level in order, chunk-boundary even
// blocks are completed in place (inline_fix) and no fix-up launch is needed;
// no CTA ever waits for another.  Each slot holds the stored factors of its
// current system and two ping-pong buffers for the transient level systems
// and right-hand sides, and is reused by the slot's next system.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "crsolve.h"
#include "cr_launch.h"

namespace crs {

struct SysDesc {
    int64_t N, offA, offB, offY;  // element offsets into the packed A, B, y / x
    int32_t m, k, mt, pad;
};

struct BatchTiles {
    int nbf[5], nbs[5], kc[5];
};

struct BatchArgs {
    const SysDesc *sys;
    const int32_t *order;
    int32_t nsys;
    int32_t *counter;
    const z2 *A, *B, *y;
    z2 *x;
    char *slots;
    int64_t slot_bytes;
    unsigned long long *status;  // [nsys]
    BatchTiles tiles;
    unsigned long long *dbg;     // bounds-checked builds: first out-of-range access
};

__host__ __device__ inline int64_t al16(int64_t b) { return (b + 15) & ~(int64_t)15; }

__host__ __device__ inline int num_levels(int64_t N) {
    int n = 1;
    while (N > 1) { N /= 2; ++n; }
    return n;
}

// Bytes of level l's stored factor region: L [no][m][m], Z [no][m][2m],
// r [no][m][k] (complex) and 1/diag(L) [no][m] (double).
__host__ __device__ inline int64_t level_region(int64_t no, int m, int k) {
    return no * (int64_t)(3 * m * m + m * k) * 16 + al16(no * (int64_t)m * 8);
}

// Slot layout of a system: the levels' factor regions, then the ping-pong
// buffers: system buffers S[p] (A then B, capacity cap[p] blocks) and vector
// buffers Y[p] (capacity cap[p] blocks of m x k), p = parity of the level
// they hold (levels 1, 3, ... in p = 1 with cap N_1; 2, 4, ... in p = 0 with cap N_2).
struct SlotLevel {
    int64_t Nl, no, ne, off;           // level sizes and the offset of its factor region
    int64_t sysbuf[2], vecbuf[2], cap[2];
};

__host__ __device__ inline int64_t slot_layout(int64_t N, int m, int k, int want, SlotLevel *out) {
    int64_t off = 0, Nl = N, N1 = N / 2, N2 = N / 4;
    const int nlev = num_levels(N);
    for (int l = 0; l < nlev; ++l) {
        const int64_t no = (Nl + 1) / 2;
        if (out && l == want) { out->Nl = Nl; out->no = no; out->ne = Nl / 2; out->off = off; }
        off += level_region(no, m, k);
        Nl /= 2;
    }
    int64_t cap[2] = {N2, N1};
    int64_t sb[2], vb[2];
    for (int p = 0; p < 2; ++p) {
        sb[p] = off;
        off += cap[p] * 2 * (int64_t)m * m * 16;
        vb[p] = off;
        off += cap[p] * (int64_t)m * k * 16;
    }
    if (out)
        for (int p = 0; p < 2; ++p) { out->sysbuf[p] = sb[p]; out->vecbuf[p] = vb[p]; out->cap[p] = cap[p]; }
    return (off + 255) & ~(int64_t)255;
}

// Level l's arguments for system d in slot `slot` (same for every thread).
__device__ inline void make_level_args(LevelArgs &a, const BatchArgs &ba, const SysDesc &d, int32_t sid, char *slot,
                                       int l) {
    const int m = d.m, k = d.k, mm = m * m, mk = m * k;
    SlotLevel sl;
    slot_layout(d.N, m, k, l, &sl);
    a = LevelArgs{};
    a.Nl = sl.Nl; a.no = sl.no; a.ne = sl.ne; a.m = m; a.k = k; a.level = l; a.inline_fix = 1;
    const int p = l & 1, q = (l + 1) & 1;
    char *reg = slot + sl.off;
    a.L = reinterpret_cast<z2 *>(reg);
    a.Z = a.L + sl.no * mm;
    a.r = a.Z + sl.no * 2 * mm;
    a.inv = reinterpret_cast<double *>(a.r + sl.no * mk);
    z2 *Sp = reinterpret_cast<z2 *>(slot + sl.sysbuf[p]), *Sq = reinterpret_cast<z2 *>(slot + sl.sysbuf[q]);
    z2 *Yp = reinterpret_cast<z2 *>(slot + sl.vecbuf[p]), *Yq = reinterpret_cast<z2 *>(slot + sl.vecbuf[q]);
    a.A = l == 0 ? ba.A + d.offA : Sp;
    a.B = l == 0 ? ba.B + d.offB : Sp + sl.cap[p] * mm;
    a.An = Sq;
    a.Bn = Sq + sl.cap[q] * mm;
    a.y = l == 0 ? ba.y + d.offY : Yp;
    a.yn = Yq;
    a.x = l == 0 ? ba.x + d.offY : Yp;
    a.xn = Yq;
    a.status = ba.status + sid;
    a.dbg = ba.dbg;
}

// The whole classic cyclic reduction of one system, run by one CTA.  The
// level arguments live in shared memory (sa) so that they do not hold
// registers across the chunk loops.
template <int MT>
__device__ __noinline__ void run_system(const BatchArgs &ba, const SysDesc &d, int32_t sid, char *slot,
                                        unsigned char *smem, LevelArgs &sa) {
    const int k = d.k;
    const int nlev = num_levels(d.N);
    const int ti = MT == 4 ? 0 : MT == 8 ? 1 : MT == 16 ? 2 : MT == 32 ? 3 : 4;
    const int nbf = ba.tiles.nbf[ti], nbs = ba.tiles.nbs[ti], kcm = ba.tiles.kc[ti];
    // down: factor level l, then reduce its right-hand side
    for (int l = 0; l < nlev; ++l) {
        if (threadIdx.x == 0) {
            make_level_args(sa, ba, d, sid, slot, l);
            sa.nb = (int)min((int64_t)nbf, sa.no);
        }
        __syncthreads();
        for (int64_t c = 0, nc = crs_num_ctas(sa.no, sa.nb); c < nc; ++c) {
            factor_chunk<MT, double>(sa, c, smem);
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            sa.nb = (int)min((int64_t)nbs, sa.no);
            sa.kc = min(kcm, k);
        }
        __syncthreads();
        const int ncc = (k + sa.kc - 1) / sa.kc;
        for (int64_t c = 0, nc = crs_num_ctas(sa.no, sa.nb); c < nc; ++c)
            for (int cc = 0; cc < ncc; ++cc) {
                solve_down_chunk<MT, double>(sa, c, cc, smem);
                __syncthreads();
            }
    }
    // up: coarsest level first
    for (int l = nlev - 1; l >= 0; --l) {
        if (threadIdx.x == 0) {
            make_level_args(sa, ba, d, sid, slot, l);
            sa.nb = (int)min((int64_t)nbs, sa.no);
            sa.kc = min(kcm, k);
        }
        __syncthreads();
        const int ncc = (k + sa.kc - 1) / sa.kc;
        for (int64_t c = 0, nc = crs_num_ctas(sa.no, sa.nb); c < nc; ++c)
            for (int cc = 0; cc < ncc; ++cc) {
                solve_up_chunk<MT, double>(sa, c, cc, smem);
                __syncthreads();
            }
    }
}

__global__ void __launch_bounds__(256, 2) k_batch(BatchArgs ba) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int32_t s_next;
    __shared__ LevelArgs s_args;
    char *slot = ba.slots + (int64_t)blockIdx.x * ba.slot_bytes;
    for (;;) {
        if (threadIdx.x == 0) s_next = atomicAdd(ba.counter, 1);
        __syncthreads();
        const int32_t i = s_next;
        __syncthreads();
        if (i >= ba.nsys) return;
        const int32_t sid = ba.order[i];
        const SysDesc d = ba.sys[sid];
        switch (d.mt) {
            case 4: run_system<4>(ba, d, sid, slot, smem_raw, s_args); break;
            case 8: run_system<8>(ba, d, sid, slot, smem_raw, s_args); break;
            case 16: run_system<16>(ba, d, sid, slot, smem_raw, s_args); break;
            case 32: run_system<32>(ba, d, sid, slot, smem_raw, s_args); break;
            default: run_system<64>(ba, d, sid, slot, smem_raw, s_args); break;
        }
        __syncthreads();
    }
}

}  // namespace crs

using crs::z2;

struct crsolve_batch_s {
    int32_t nsys = 0;
    std::vector<crs::SysDesc> sys;
    std::vector<int32_t> order;
    crs::BatchTiles tiles{};
    int threads = 256, device = 0, nsm = 0;
    int64_t slot_bytes = 0, nA = 0, nB = 0, nY = 0;
    int32_t nslots = 0;
    size_t smem = 0;
    size_t offSys = 0, offOrder = 0, offCounter = 0, offStatus = 0, offDbg = 0, offSlots = 0, total = 0;
    char *ws = nullptr;
    bool uploaded = false;
    cudaGraphExec_t gexec = nullptr;
    cudaGraph_t graph = nullptr;
    const void *gptr[4] = {nullptr, nullptr, nullptr, nullptr};
};

namespace {

const int kMtList[5] = {4, 8, 16, 32, 64};

// Largest dynamic shared memory k_batch may use: the device's opt-in limit
// minus the kernel's static shared memory; also raises the kernel's limit.
int batch_smem_limit(int device, size_t *limit) {
    int optin = 0;
    cudaFuncAttributes fa{};
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device) != cudaSuccess ||
        cudaFuncGetAttributes(&fa, crs::k_batch) != cudaSuccess)
        return CRSOLVE_ECUDA;
    const int dyn = optin - (int)fa.sharedSizeBytes;
    if (dyn <= 0 || cudaFuncSetAttribute(crs::k_batch, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) != cudaSuccess)
        return CRSOLVE_ECUDA;
    *limit = (size_t)dyn;
    return CRSOLVE_OK;
}

size_t batch_smem(const crsolve_batch_s *b) {
    size_t smem = 0;
    bool present[5] = {false, false, false, false, false};
    for (const auto &d : b->sys) present[d.mt == 4 ? 0 : d.mt == 8 ? 1 : d.mt == 16 ? 2 : d.mt == 32 ? 3 : 4] = true;
    for (int i = 0; i < 5; ++i) {
        if (!present[i]) continue;
        smem = std::max(smem, crs::factor_smem_bytes(kMtList[i], b->tiles.nbf[i], 8));
        smem = std::max(smem, crs::solve_smem_bytes(kMtList[i], b->tiles.nbs[i], b->tiles.kc[i], 3, 8));
    }
    return smem;
}

void release_graph(crsolve_batch_s *b) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
}

// Workspace: descriptors, order, counter, per-system status, then the slots.
void layout(crsolve_batch_s *b, int32_t nslots) {
    size_t cur = 0;
    auto take = [&](size_t bytes) { size_t o = cur; cur += (bytes + 255) & ~(size_t)255; return o; };
    b->offSys = take(b->sys.size() * sizeof(crs::SysDesc));
    b->offOrder = take(b->order.size() * sizeof(int32_t));
    b->offCounter = take(sizeof(int32_t));
    b->offStatus = take(b->sys.size() * sizeof(unsigned long long));
    b->offDbg = take(sizeof(unsigned long long));
    b->offSlots = take(0);
    b->nslots = nslots;
    b->total = b->offSlots + (size_t)nslots * (size_t)b->slot_bytes;
}

int enqueue(crsolve_batch_s *b, const z2 *A, const z2 *B, const z2 *y, z2 *x, cudaStream_t s) {
    if (cudaMemsetAsync(b->ws + b->offCounter, 0, sizeof(int32_t), s) != cudaSuccess) return CRSOLVE_ECUDA;
    if (cudaMemsetAsync(b->ws + b->offStatus, 0xFF, b->sys.size() * sizeof(unsigned long long), s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    crs::BatchArgs ba{};
    ba.sys = reinterpret_cast<const crs::SysDesc *>(b->ws + b->offSys);
    ba.order = reinterpret_cast<const int32_t *>(b->ws + b->offOrder);
    ba.nsys = b->nsys;
    ba.counter = reinterpret_cast<int32_t *>(b->ws + b->offCounter);
    ba.A = A; ba.B = B; ba.y = y; ba.x = x;
    ba.slots = b->ws + b->offSlots;
    ba.slot_bytes = b->slot_bytes;
    ba.status = reinterpret_cast<unsigned long long *>(b->ws + b->offStatus);
    ba.tiles = b->tiles;
    ba.dbg = reinterpret_cast<unsigned long long *>(b->ws + b->offDbg);
#ifdef CRSOLVE_DEBUG_BOUNDS
    if (cudaMemsetAsync(ba.dbg, 0xFF, sizeof(unsigned long long), s) != cudaSuccess) return CRSOLVE_ECUDA;
#endif
    crs::k_batch<<<b->nslots, b->threads, b->smem, s>>>(ba);
    return cudaGetLastError() == cudaSuccess ? CRSOLVE_OK : CRSOLVE_ECUDA;
}

int prepare(crsolve_batch_s *b) {
    if (b->uploaded) return CRSOLVE_OK;
    size_t limit = 0;
    int rc = batch_smem_limit(b->device, &limit);
    if (rc) return rc;
    if (b->smem > limit) return CRSOLVE_EINVAL;
    if (cudaMemcpy(b->ws + b->offSys, b->sys.data(), b->sys.size() * sizeof(crs::SysDesc), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->ws + b->offOrder, b->order.data(), b->order.size() * sizeof(int32_t), cudaMemcpyHostToDevice) !=
            cudaSuccess)
        return CRSOLVE_ECUDA;
    b->uploaded = true;
    return CRSOLVE_OK;
}

bool ok_ptrs(const crsolve_batch_s *b, const void *A, const void *B, const void *y, const void *x) {
    if (!A || !y || !x || (b->nB > 0 && !B)) return false;
    return ((((uintptr_t)A | (uintptr_t)B | (uintptr_t)y | (uintptr_t)x) & 15u) == 0) && x != y;
}

}  // namespace

extern "C" {

int crsolve_batch_create(int32_t nsys, const int64_t *N, const int32_t *m, const int32_t *k, crsolve_batch *out) {
    if (!out) return CRSOLVE_EINVAL;
    *out = nullptr;
    if (nsys < 1 || !N || !m || !k) return CRSOLVE_EINVAL;
    for (int32_t i = 0; i < nsys; ++i) {
        if (N[i] < 1 || m[i] < 1 || k[i] < 1) return CRSOLVE_EINVAL;
        if (m[i] > CRSOLVE_MAX_M || k[i] > CRSOLVE_MAX_K) return CRSOLVE_EUNSUPPORTED;
    }
    crsolve_batch_s *b = new (std::nothrow) crsolve_batch_s();
    if (!b) return CRSOLVE_ENOMEM;
    b->nsys = nsys;
    b->sys.resize(nsys);
    std::vector<double> cost(nsys);
    int64_t oA = 0, oB = 0, oY = 0;
    for (int32_t i = 0; i < nsys; ++i) {
        crs::SysDesc &d = b->sys[i];
        d.N = N[i]; d.m = m[i]; d.k = k[i]; d.mt = crs::pick_mt(m[i]); d.pad = 0;
        d.offA = oA; d.offB = oB; d.offY = oY;
        oA += N[i] * (int64_t)m[i] * m[i];
        oB += (N[i] - 1) * (int64_t)m[i] * m[i];
        oY += N[i] * (int64_t)m[i] * k[i];
        const double md = m[i];
        cost[i] = (double)N[i] * (25.33 * md * md * md + 40.0 * md * md * k[i]);
        b->slot_bytes = std::max(b->slot_bytes, crs::slot_layout(N[i], m[i], k[i], -1, nullptr));
    }
    b->nA = oA; b->nB = oB; b->nY = oY;
    b->order.resize(nsys);
    std::iota(b->order.begin(), b->order.end(), 0);
    std::stable_sort(b->order.begin(), b->order.end(), [&](int32_t a, int32_t c) { return cost[a] > cost[c]; });
    // default tiles per block-size class: odd blocks per chunk (factor, solve), rhs columns
    const int nbf[5] = {16, 8, 4, 2, 1}, nbs[5] = {16, 8, 4, 2, 1}, kc[5] = {16, 16, 16, 16, 16};
    for (int i = 0; i < 5; ++i) { b->tiles.nbf[i] = nbf[i]; b->tiles.nbs[i] = nbs[i]; b->tiles.kc[i] = kc[i]; }
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device) != cudaSuccess) {
        delete b;
        return CRSOLVE_ECUDA;
    }
    b->smem = batch_smem(b);
    *out = b;
    return CRSOLVE_OK;
}

int crsolve_batch_tile_set(crsolve_batch b, int32_t mt, int32_t nb_factor, int32_t nb_solve, int32_t kc) {
    if (!b || b->ws) return CRSOLVE_EINVAL;
    int i = -1;
    for (int j = 0; j < 5; ++j)
        if (kMtList[j] == mt) i = j;
    if (i < 0 || nb_factor < 1 || nb_solve < 1 || kc < 1 || kc > CRSOLVE_MAX_K) return CRSOLVE_EINVAL;
    b->tiles.nbf[i] = nb_factor; b->tiles.nbs[i] = nb_solve; b->tiles.kc[i] = kc;
    b->smem = batch_smem(b);
    size_t limit = 0;
    const int rc = batch_smem_limit(b->device, &limit);
    if (rc) return rc;
    return b->smem <= limit ? CRSOLVE_OK : CRSOLVE_EINVAL;
}

int crsolve_batch_workspace_bytes(crsolve_batch b, size_t max_bytes, size_t *bytes, int32_t *nslots) {
    if (!b || !bytes) return CRSOLVE_EINVAL;
    int per_sm = 0;
    size_t limit = 0;
    int rc = batch_smem_limit(b->device, &limit);
    if (rc) return rc;
    if (b->smem > limit) return CRSOLVE_EINVAL;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, crs::k_batch, b->threads, b->smem) != cudaSuccess)
        return CRSOLVE_ECUDA;
    if (per_sm < 1) return CRSOLVE_EINVAL;
    int64_t want = std::min<int64_t>((int64_t)per_sm * b->nsm, b->nsys);
    layout(b, 0);
    if (max_bytes) {
        const int64_t fit = ((int64_t)max_bytes - (int64_t)b->offSlots) / b->slot_bytes;
        if (fit < 1) return CRSOLVE_ENOMEM;
        want = std::min(want, fit);
    }
    layout(b, (int32_t)want);
    *bytes = b->total;
    if (nslots) *nslots = b->nslots;
    return CRSOLVE_OK;
}

int crsolve_batch_set_workspace(crsolve_batch b, void *dev_ptr, size_t bytes) {
    if (!b || !dev_ptr || ((uintptr_t)dev_ptr & 255u) || b->nslots < 1) return CRSOLVE_EINVAL;
    if (bytes < b->total) return CRSOLVE_ENOMEM;
    b->ws = static_cast<char *>(dev_ptr);
    b->uploaded = false;
    release_graph(b);
    return CRSOLVE_OK;
}

int crsolve_batch_offsets(crsolve_batch b, int64_t *offA, int64_t *offB, int64_t *offY, int64_t *totals) {
    if (!b) return CRSOLVE_EINVAL;
    for (int32_t i = 0; i < b->nsys; ++i) {
        if (offA) offA[i] = b->sys[i].offA;
        if (offB) offB[i] = b->sys[i].offB;
        if (offY) offY[i] = b->sys[i].offY;
    }
    if (totals) { totals[0] = b->nA; totals[1] = b->nB; totals[2] = b->nY; }
    return CRSOLVE_OK;
}

int crsolve_batch_solve(crsolve_batch b, const crsolve_z *A, const crsolve_z *B, const crsolve_z *y, crsolve_z *x,
                        void *stream) {
    if (!b || !ok_ptrs(b, A, B, y, x)) return CRSOLVE_EINVAL;
    if (!b->ws) return CRSOLVE_ENOMEM;
    int rc = prepare(b);
    if (rc) return rc;
    return enqueue(b, reinterpret_cast<const z2 *>(A), reinterpret_cast<const z2 *>(B),
                   reinterpret_cast<const z2 *>(y), reinterpret_cast<z2 *>(x), static_cast<cudaStream_t>(stream));
}

int crsolve_batch_graph_launch(crsolve_batch b, const crsolve_z *A, const crsolve_z *B, const crsolve_z *y,
                               crsolve_z *x, void *stream) {
    if (!b || !ok_ptrs(b, A, B, y, x)) return CRSOLVE_EINVAL;
    if (!b->ws) return CRSOLVE_ENOMEM;
    int rc = prepare(b);
    if (rc) return rc;
    const void *ptrs[4] = {A, B, y, x};
    if (!b->gexec || memcmp(ptrs, b->gptr, sizeof(ptrs)) != 0) {
        release_graph(b);
        cudaStream_t cs;
        if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) return CRSOLVE_ECUDA;
        rc = CRSOLVE_OK;
        if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) rc = CRSOLVE_ECUDA;
        if (!rc) rc = enqueue(b, reinterpret_cast<const z2 *>(A), reinterpret_cast<const z2 *>(B),
                              reinterpret_cast<const z2 *>(y), reinterpret_cast<z2 *>(x), cs);
        cudaGraph_t g = nullptr;
        if (cudaStreamEndCapture(cs, &g) != cudaSuccess && !rc) rc = CRSOLVE_ECUDA;
        cudaStreamDestroy(cs);
        if (!rc && cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) rc = CRSOLVE_ECUDA;
        b->graph = g;
        if (rc) { release_graph(b); return rc; }
        memcpy(b->gptr, ptrs, sizeof(ptrs));
    }
    return cudaGraphLaunch(b->gexec, static_cast<cudaStream_t>(stream)) == cudaSuccess ? CRSOLVE_OK : CRSOLVE_ECUDA;
}

int crsolve_batch_debug_bounds(crsolve_batch b, uint64_t *record, void *stream) {
    if (!b || !record) return CRSOLVE_EINVAL;
#ifdef CRSOLVE_DEBUG_BOUNDS
    if (!b->ws) return CRSOLVE_ENOMEM;
    unsigned long long v = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(&v, b->ws + b->offDbg, sizeof(v), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
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

int crsolve_batch_info(crsolve_batch b, crsolve_info *out, void *stream) {
    if (!b || !out) return CRSOLVE_EINVAL;
    if (!b->ws) return CRSOLVE_ENOMEM;
    std::vector<unsigned long long> st(b->nsys);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaMemcpyAsync(st.data(), b->ws + b->offStatus, st.size() * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return CRSOLVE_ECUDA;
    for (int32_t i = 0; i < b->nsys; ++i) {
        if (st[i] == CRS_NO_FAIL) {
            out[i] = crsolve_info{CRSOLVE_OK, 0, 0, 0};
        } else {
            const int level = (int)(st[i] >> 40);
            const int64_t block = (int64_t)(st[i] & ((1ull << 40) - 1));
            out[i] = crsolve_info{CRSOLVE_NOT_PD, level, block, block << level};
        }
    }
    return CRSOLVE_OK;
}

int crsolve_batch_destroy(crsolve_batch b) {
    if (!b) return CRSOLVE_EINVAL;
    release_graph(b);
    delete b;
    return CRSOLVE_OK;
}

}  // extern "C"
