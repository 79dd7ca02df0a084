// cr_solve32.cu -- the down and up sweeps of the FP32 levels of the
// mixed-precision form for blocks of 33..64 rows (class MT = 64), written as
// complex matrix products.
//
// The FP32 factorisation of this class keeps Linv = L^{-1} (lower triangular,
// computed in the same blocked substitution as Z = L^{-1} [B | B^H]) in place
// of L.  A level's two sweeps (Sec. 2, eq. Formulas) then need no
// substitution chain:
//   down:  r = Linv y_odd,  u = Z^H r = [P^H r ; Q^H r],
//          v_t = y_even - Q^H r  (P^H r goes to the left even block)
//   up:    w = r - Z [x_left ; x_right],  x_odd = Linv^H w
// Each sweep is two dense products whose outputs are all independent, with
// the flop count of the substitutions they replace.
//
// GPU mapping.  Persistent CTAs of 256 threads, one per SM.  A work item is
// one odd block t and one chunk of KC right-hand-side columns.  Its operands
// are copied into shared memory with cp.async in two groups, the operands of
// the first product and those of the second; the next item's group is issued
// as soon as the buffers it fills are free, so the copies of one product
// overlap the arithmetic of the other.  Each thread owns RP consecutive rows
// x RC columns of a product in registers; per step of the reduction it loads
// RP matrix entries (shared by the threads of the same rows) and RC vector
// entries (shared by the threads of the same columns).  Matrix rows are
// padded by 16 bytes in shared memory, so that the rows a warp reads at one
// step fall into different banks.
#include "cr_launch.h"

namespace crs {

namespace {

constexpr int kGMT = 64;                 // block rows of the class
constexpr int kGLdL = kGMT + 2;          // Linv row in shared memory (complex)
constexpr int kGLdZ = 2 * kGMT + 2;      // Z row in shared memory (complex)
constexpr int kGThreads = 256;

__device__ __forceinline__ void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Copy rows x cols complex values, row stride lds in global memory, into
// shared memory with row stride ldd.  `wide`: 16-byte copies (cols, lds and
// the source offset even), else 8-byte ones.  inb(i) is the bounds check of
// element i of the source (a no-op outside bounds-checked builds); an element
// that fails it is not copied.
template <class InB>
__device__ __forceinline__ void copy_tile(c2 *dst, int ldd, const c2 *src, int64_t lds, int rows, int cols, bool wide,
                                          InB inb) {
    const int tid = threadIdx.x;
    if (wide) {
        const int gpr = cols >> 1;
        for (int e = tid; e < rows * gpr; e += kGThreads) {
            const int r = e / gpr, g = e - r * gpr;
            const int64_t i = r * lds + 2 * g;
            if (inb(i) && inb(i + 1)) cp_async16(dst + r * ldd + 2 * g, src + i);
        }
    } else {
        for (int e = tid; e < rows * cols; e += kGThreads) {
            const int r = e / cols, c = e - r * cols;
            const int64_t i = r * lds + c;
            if (inb(i)) cp_async8(dst + r * ldd + c, src + i);
        }
    }
}

__device__ __forceinline__ void cfma(c2 &acc, c2 a, c2 b) {   // acc += a b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(-a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(a.y, b.x, acc.y);
}
__device__ __forceinline__ void cfma_ca(c2 &acc, c2 a, c2 b) {   // acc += conj(a) b
    acc.x = fmaf(a.x, b.x, acc.x);
    acc.x = fmaf(a.y, b.y, acc.x);
    acc.y = fmaf(a.x, b.y, acc.y);
    acc.y = fmaf(-a.y, b.x, acc.y);
}

// Thread tile of the products for a chunk of KC columns: RC columns per
// thread (two pairs {2cg, 2cg+1} and {KC/2 + 2cg, KC/2 + 2cg + 1}, or one
// pair when RC = 2), CG column groups, RG row groups of 256 / CG threads.
template <int KC>
struct GTile {
    static constexpr int RC = KC >= 16 ? 4 : 2;
    static constexpr int CG = KC / RC;
    static constexpr int RG = kGThreads / CG;
    __device__ static int col(int cg, int q) { return (q < 2 ? 0 : KC / 2) + 2 * cg + (q & 1); }
};

// The RC vector entries of row s of a [rows][KC] panel for column group cg.
template <int KC>
__device__ __forceinline__ void load_vec(const c2 *V, int s, int cg, c2 (&v)[GTile<KC>::RC]) {
    const float4 a = *reinterpret_cast<const float4 *>(V + s * KC + 2 * cg);
    v[0] = make_float2(a.x, a.y);
    v[1] = make_float2(a.z, a.w);
    if constexpr (GTile<KC>::RC == 4) {
        const float4 b = *reinterpret_cast<const float4 *>(V + s * KC + KC / 2 + 2 * cg);
        v[2] = make_float2(b.x, b.y);
        v[3] = make_float2(b.z, b.w);
    }
}

// acc[j][q] += M(p0 + j, s) V[s][col q] for s in [s0, s1), with M(p, s) the
// entry (p, s) of a row-major matrix Mb with row stride ldm (even).
template <int KC, int RP>
__device__ __forceinline__ void gemm_rows(c2 (&acc)[RP][GTile<KC>::RC], const c2 *Mb, int ldm, int p0, const c2 *V,
                                          int cg, int s0, int s1) {
    constexpr int RC = GTile<KC>::RC;
    int s = s0;
    for (; s + 1 < s1; s += 2) {
        c2 v0[RC], v1[RC];
        load_vec<KC>(V, s, cg, v0);
        load_vec<KC>(V, s + 1, cg, v1);
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const float4 mm = *reinterpret_cast<const float4 *>(Mb + (p0 + j) * ldm + s);
            const c2 a0 = make_float2(mm.x, mm.y), a1 = make_float2(mm.z, mm.w);
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                cfma(acc[j][q], a0, v0[q]);
                cfma(acc[j][q], a1, v1[q]);
            }
        }
    }
    if (s < s1) {
        c2 v0[RC];
        load_vec<KC>(V, s, cg, v0);
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const c2 a0 = Mb[(p0 + j) * ldm + s];
#pragma unroll
            for (int q = 0; q < RC; ++q) cfma(acc[j][q], a0, v0[q]);
        }
    }
}

// acc[j][q] += conj(M(s, p0 + j)) V[s][col q] for s in [s0, s1): the
// conjugate transpose of a row-major matrix Mb with row stride ldm (even).
template <int KC, int RP>
__device__ __forceinline__ void gemm_cols_h(c2 (&acc)[RP][GTile<KC>::RC], const c2 *Mb, int ldm, int p0, const c2 *V,
                                            int cg, int s0, int s1) {
    constexpr int RC = GTile<KC>::RC;
#pragma unroll 2
    for (int s = s0; s < s1; ++s) {
        c2 v[RC], a[RP];
        load_vec<KC>(V, s, cg, v);
        if constexpr (RP == 1) {
            a[0] = Mb[s * ldm + p0];
        } else {
#pragma unroll
            for (int j = 0; j < RP; j += 2) {
                const float4 mm = *reinterpret_cast<const float4 *>(Mb + s * ldm + p0 + j);
                a[j] = make_float2(mm.x, mm.y);
                a[j + 1] = make_float2(mm.z, mm.w);
            }
        }
#pragma unroll
        for (int j = 0; j < RP; ++j)
#pragma unroll
            for (int q = 0; q < RC; ++q) cfma_ca(acc[j][q], a[j], v[q]);
    }
}

template <int KC>
constexpr size_t gsmem_bytes() {
    return (size_t)(kGMT * kGLdL + kGMT * kGLdZ + 3 * kGMT * KC) * sizeof(c2);
}

// ------------------------------------------------------------------ down

// Shared memory: sLi [64][66], sZ [64][130], sY (y_odd), sYe (y_even), sR
// (r), each [64][KC].  Group A of an item: Linv, y_odd; group B: Z, y_even.
template <int KC>
__global__ void __launch_bounds__(kGThreads, 1) k_solve_down_g32(LevelArgsT<float> a) {
    using T = GTile<KC>;
    constexpr int RC = T::RC, CG = T::CG, RG = T::RG;
    constexpr int RPA = kGMT / RG, RPB = 2 * kGMT / RG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2 *sLi = reinterpret_cast<c2 *>(smem_raw);
    c2 *sZ = sLi + kGMT * kGLdL;
    c2 *sY = sZ + kGMT * kGLdZ;
    c2 *sYe = sY + kGMT * KC;
    c2 *sR = sYe + kGMT * KC;

    const int m = a.m, k = a.k, tid = threadIdx.x, warp = tid >> 5;
    const int64_t mm = (int64_t)m * m, mk = (int64_t)m * k;
    const int nch = (k + KC - 1) / KC;
    const int64_t items = a.no * nch;
    const int cg = tid % CG, rg = tid / CG;
    const bool wideL = (m & 1) == 0, wideV = (k & 1) == 0;

    auto issue_a = [&](int64_t it) {
        const int64_t t = it / nch;
        const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
        copy_tile(sLi, kGLdL, a.L + t * mm, m, m, m, wideL,
                  [&](int64_t i) { return CRS_IN(a, kDbgL, t * mm + i); });
        copy_tile(sY, KC, a.y + 2 * t * mk + c0, k, m, kw, wideV,
                  [&](int64_t i) { return CRS_IN(a, kDbgY, 2 * t * mk + c0 + i); });
        cp_async_commit();
    };
    auto issue_b = [&](int64_t it) {
        const int64_t t = it / nch;
        const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
        copy_tile(sZ, kGLdZ, a.Z + t * 2 * mm, 2 * m, m, 2 * m, true,
                  [&](int64_t i) { return CRS_IN(a, kDbgZ, t * 2 * mm + i); });
        if (t < a.ne)
            copy_tile(sYe, KC, a.y + (2 * t + 1) * mk + c0, k, m, kw, wideV,
                      [&](int64_t i) { return CRS_IN(a, kDbgY, (2 * t + 1) * mk + c0 + i); });
        cp_async_commit();
    };

    int64_t it = blockIdx.x;
    if (it >= items) return;
    issue_a(it);
    issue_b(it);
    for (; it < items; it += gridDim.x) {
        const int64_t t = it / nch, nxt = it + gridDim.x;
        const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);

        // r = Linv y_odd (Linv lower triangular: a warp's rows end at row
        // (warp + 1) * rows-per-warp - 1, so its reduction stops there)
        cp_async_wait<1>();
        __syncthreads();
        c2 ra[RPA][RC];
#pragma unroll
        for (int j = 0; j < RPA; ++j)
#pragma unroll
            for (int q = 0; q < RC; ++q) ra[j][q] = make_float2(0.f, 0.f);
        const int s1a = min(m, (warp + 1) * (32 / CG) * RPA);
        gemm_rows<KC, RPA>(ra, sLi, kGLdL, rg * RPA, sY, cg, 0, s1a);
        __syncthreads();   // Linv and y_odd read: the next item's group A may land
        if (nxt < items) issue_a(nxt);
        else cp_async_commit();
#pragma unroll
        for (int j = 0; j < RPA; ++j) {
            const int i = rg * RPA + j;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const int c = T::col(cg, q);
                sR[i * KC + c] = ra[j][q];
                if (i < m && c < kw && CRS_IN(a, kDbgR, t * mk + i * k + c0 + c)) a.r[t * mk + i * k + c0 + c] = ra[j][q];
            }
        }

        // u = Z^H r: rows p < m are P^H r (to the chunk-boundary buffer of
        // this block, subtracted from the left even block by the fix-up),
        // rows m <= p < 2m are Q^H r (v_t = y_even - Q^H r)
        cp_async_wait<1>();
        __syncthreads();
        c2 ub[RPB][RC];
#pragma unroll
        for (int j = 0; j < RPB; ++j)
#pragma unroll
            for (int q = 0; q < RC; ++q) ub[j][q] = make_float2(0.f, 0.f);
        gemm_cols_h<KC, RPB>(ub, sZ, kGLdZ, rg * RPB, sR, cg, 0, m);
#pragma unroll
        for (int j = 0; j < RPB; ++j) {
            const int p = rg * RPB + j;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const int c = T::col(cg, q);
                if (c >= kw) continue;
                if (p < m) {
                    if (t >= 1 && CRS_IN(a, kDbgCbd, t * mk + p * k + c0 + c)) a.cbd[t * mk + p * k + c0 + c] = ub[j][q];
                } else if (p < 2 * m && t < a.ne) {
                    const int i = p - m;
                    if (CRS_IN(a, kDbgYn, t * mk + i * k + c0 + c))
                        a.yn[t * mk + i * k + c0 + c] = zsub(sYe[i * KC + c], ub[j][q]);
                }
            }
        }
        __syncthreads();   // Z, r and y_even read: the next item's group B may land
        if (nxt < items) issue_b(nxt);
        else cp_async_commit();
    }
    cp_async_wait<0>();
}

// -------------------------------------------------------------------- up

// Shared memory: sZ [64][130], sLi [64][66], sR (r, then w) [64][KC], sX
// ([x_left; x_right]) [128][KC].  Group A of an item: Z, x_left, x_right;
// group B: Linv, r.
template <int KC>
__global__ void __launch_bounds__(kGThreads, 1) k_solve_up_g32(LevelArgsT<float> a) {
    using T = GTile<KC>;
    constexpr int RC = T::RC, CG = T::CG, RG = T::RG;
    constexpr int RP = kGMT / RG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2 *sZ = reinterpret_cast<c2 *>(smem_raw);
    c2 *sLi = sZ + kGMT * kGLdZ;
    c2 *sR = sLi + kGMT * kGLdL;
    c2 *sX = sR + kGMT * KC;

    const int m = a.m, k = a.k, tid = threadIdx.x, warp = tid >> 5;
    const int64_t mm = (int64_t)m * m, mk = (int64_t)m * k;
    const int nch = (k + KC - 1) / KC;
    const int64_t items = a.no * nch;
    const int cg = tid % CG, rg = tid / CG;
    const bool wideL = (m & 1) == 0, wideV = (k & 1) == 0;

    if (a.level == 0 && *a.status != CRS_NO_FAIL) {
        // the factorisation broke down: the result is NaN
        const c2 nan2 = make_float2(qnan(0.f), qnan(0.f));
        for (int64_t e = blockIdx.x * (int64_t)kGThreads + tid; e < a.Nl * mk; e += (int64_t)gridDim.x * kGThreads)
            if (CRS_IN(a, kDbgX, e)) a.x[e] = nan2;
        return;
    }

    auto issue_a = [&](int64_t it) {
        const int64_t t = it / nch;
        const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
        copy_tile(sZ, kGLdZ, a.Z + t * 2 * mm, 2 * m, m, 2 * m, true,
                  [&](int64_t i) { return CRS_IN(a, kDbgZ, t * 2 * mm + i); });
        // [x_left; x_right] = [xn_{t-1}; xn_t], zero past either end
        if (t >= 1)
            copy_tile(sX, KC, a.xn + (t - 1) * mk + c0, k, m, kw, wideV,
                      [&](int64_t i) { return CRS_IN(a, kDbgXn, (t - 1) * mk + c0 + i); });
        else
            for (int e = tid; e < m * KC; e += kGThreads) sX[e] = make_float2(0.f, 0.f);
        if (t < a.ne)
            copy_tile(sX + m * KC, KC, a.xn + t * mk + c0, k, m, kw, wideV,
                      [&](int64_t i) { return CRS_IN(a, kDbgXn, t * mk + c0 + i); });
        else
            for (int e = tid; e < m * KC; e += kGThreads) sX[m * KC + e] = make_float2(0.f, 0.f);
        cp_async_commit();
    };
    auto issue_b = [&](int64_t it) {
        const int64_t t = it / nch;
        const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
        copy_tile(sLi, kGLdL, a.L + t * mm, m, m, m, wideL,
                  [&](int64_t i) { return CRS_IN(a, kDbgL, t * mm + i); });
        copy_tile(sR, KC, a.r + t * mk + c0, k, m, kw, wideV,
                  [&](int64_t i) { return CRS_IN(a, kDbgR, t * mk + c0 + i); });
        cp_async_commit();
    };

    int64_t it = blockIdx.x;
    if (it >= items) return;
    issue_a(it);
    issue_b(it);
    for (; it < items; it += gridDim.x) {
        const int64_t t = it / nch, nxt = it + gridDim.x;
        const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);

        // Z [x_left; x_right]
        cp_async_wait<1>();
        __syncthreads();
        if (t < a.ne) {
            // the even unknowns of this level are the next level's
            for (int e = tid; e < m * kw; e += kGThreads) {
                const int i = e / kw, c = e - i * kw;
                if (CRS_IN(a, kDbgX, (2 * t + 1) * mk + i * k + c0 + c))
                    a.x[(2 * t + 1) * mk + i * k + c0 + c] = sX[(m + i) * KC + c];
            }
        }
        c2 acc[RP][RC];
#pragma unroll
        for (int j = 0; j < RP; ++j)
#pragma unroll
            for (int q = 0; q < RC; ++q) acc[j][q] = make_float2(0.f, 0.f);
        gemm_rows<KC, RP>(acc, sZ, kGLdZ, rg * RP, sX, cg, 0, 2 * m);
        __syncthreads();   // Z and x read: the next item's group A may land
        if (nxt < items) issue_a(nxt);
        else cp_async_commit();

        // w = r - Z [x_left; x_right], in place of r (each thread its own
        // entries, after every thread's copies of r have landed)
        cp_async_wait<1>();
        __syncthreads();
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const int i = rg * RP + j;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const int c = T::col(cg, q);
                sR[i * KC + c] = zsub(sR[i * KC + c], acc[j][q]);
            }
        }
        __syncthreads();

        // x_odd = Linv^H w (Linv^H upper triangular: a warp's rows start at
        // row warp * rows-per-warp, so its reduction starts there)
#pragma unroll
        for (int j = 0; j < RP; ++j)
#pragma unroll
            for (int q = 0; q < RC; ++q) acc[j][q] = make_float2(0.f, 0.f);
        gemm_cols_h<KC, RP>(acc, sLi, kGLdL, rg * RP, sR, cg, min(m, warp * (32 / CG) * RP), m);
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const int i = rg * RP + j;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const int c = T::col(cg, q);
                if (i < m && c < kw && CRS_IN(a, kDbgX, 2 * t * mk + i * k + c0 + c))
                    a.x[2 * t * mk + i * k + c0 + c] = acc[j][q];
            }
        }
        __syncthreads();   // Linv and w read: the next item's group B may land
        if (nxt < items) issue_b(nxt);
        else cp_async_commit();
    }
    cp_async_wait<0>();
}

int g32_sms() {
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return 1;
    return n > 0 ? n : 1;
}

template <int KC>
cudaError_t down_g32(const LevelArgsT<float> &a, cudaStream_t s) {
    const int64_t items = a.no * ((a.k + KC - 1) / KC);
    if (items < 1) return cudaSuccess;
    const unsigned grid = (unsigned)(items < g32_sms() ? items : g32_sms());
    k_solve_down_g32<KC><<<grid, kGThreads, gsmem_bytes<KC>(), s>>>(a);
    return cudaGetLastError();
}

template <int KC>
cudaError_t up_g32(const LevelArgsT<float> &a, cudaStream_t s) {
    const int64_t items = a.no * ((a.k + KC - 1) / KC);
    if (items < 1) return cudaSuccess;
    const unsigned grid = (unsigned)(items < g32_sms() ? items : g32_sms());
    k_solve_up_g32<KC><<<grid, kGThreads, gsmem_bytes<KC>(), s>>>(a);
    return cudaGetLastError();
}

template <int KC>
cudaError_t prepare_g32_kc(int optin) {
    const int need = (int)gsmem_bytes<KC>();
    if (need > optin) return cudaErrorInvalidValue;
    cudaError_t e = cudaFuncSetAttribute(k_solve_down_g32<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_solve_up_g32<KC>, cudaFuncAttributeMaxDynamicSharedMemorySize, need);
}

}  // namespace

int solve_kc_g32(int k) { return k <= 8 ? 8 : (k <= 16 ? 16 : 32); }

cudaError_t prepare_solve_g32(int optin) {
    cudaError_t e = prepare_g32_kc<8>(optin);
    if (e == cudaSuccess) e = prepare_g32_kc<16>(optin);
    if (e == cudaSuccess) e = prepare_g32_kc<32>(optin);
    return e;
}

cudaError_t launch_solve_down_g32(const LevelArgsT<float> &a, cudaStream_t s) {
    if (a.m > kGMT || a.m < 1 || a.nb != 1 || a.kc != solve_kc_g32(a.k)) return cudaErrorInvalidValue;
    switch (a.kc) {
        case 8: return down_g32<8>(a, s);
        case 16: return down_g32<16>(a, s);
        default: return down_g32<32>(a, s);
    }
}

cudaError_t launch_solve_up_g32(const LevelArgsT<float> &a, cudaStream_t s) {
    if (a.m > kGMT || a.m < 1 || a.nb != 1 || a.kc != solve_kc_g32(a.k)) return cudaErrorInvalidValue;
    switch (a.kc) {
        case 8: return up_g32<8>(a, s);
        case 16: return up_g32<16>(a, s);
        default: return up_g32<32>(a, s);
    }
}

}  // namespace crs
