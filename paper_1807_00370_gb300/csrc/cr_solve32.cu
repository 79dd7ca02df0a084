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
// are copied into shared memory with cp.async in groups that are issued as
// soon as the buffers they fill are free: Z (64 KB, the operand of the larger
// product of either sweep) is double-buffered and requested two items ahead,
// the other operands one product ahead, so the copies overlap the
// arithmetic.  Each thread owns RP consecutive rows x RC columns of a product
// in registers (up to 4 x 4: 32 row groups x 8 column groups, or 16 x 8 in
// each half of the CTA when the two halves split the reduction); per step of
// the reduction it loads RP matrix entries (shared by the threads of the
// same rows) and RC vector entries (shared by the threads of the same
// columns), so that the shared-memory loads stay well below the FMAs.  Matrix rows
// are padded by 16 bytes in shared memory, so that the rows a warp reads at
// one step fall into different banks.
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

// Thread tile of the products for a chunk of KC columns: CG = 8 column
// groups of RC = KC / 8 columns ({2cg, 2cg+1, KC/2 + 2cg, KC/2 + 2cg + 1},
// {2cg, 2cg+1} or {cg}), RG = 32 row groups.
template <int KC>
struct GTile {
    static constexpr int CG = 8;
    static constexpr int RC = KC / CG;
    static constexpr int RG = kGThreads / CG;
    __device__ static int col(int cg, int q) {
        if constexpr (RC == 4) return (q < 2 ? 0 : KC / 2) + 2 * cg + (q & 1);
        else if constexpr (RC == 2) return 2 * cg + q;
        else return cg;
    }
};

// The RC vector entries of row s of a [rows][KC] panel for column group cg.
template <int KC>
__device__ __forceinline__ void load_vec(const c2 *V, int s, int cg, c2 (&v)[GTile<KC>::RC]) {
    if constexpr (GTile<KC>::RC == 1) {
        v[0] = V[s * KC + cg];
    } else {
        const float4 a = *reinterpret_cast<const float4 *>(V + s * KC + 2 * cg);
        v[0] = make_float2(a.x, a.y);
        v[1] = make_float2(a.z, a.w);
        if constexpr (GTile<KC>::RC == 4) {
            const float4 b = *reinterpret_cast<const float4 *>(V + s * KC + KC / 2 + 2 * cg);
            v[2] = make_float2(b.x, b.y);
            v[3] = make_float2(b.z, b.w);
        }
    }
}

// acc[j][q] += M(p0 + j, s) V[s][col q] for s in [s0, s1), with M(p, s) the
// entry (p, s) of a row-major matrix Mb with row stride ldm (even).
template <int KC, int RP>
__device__ __forceinline__ void gemm_rows(c2 (&acc)[RP][GTile<KC>::RC], const c2 *Mb, int ldm, int p0, const c2 *V,
                                          int cg, int s0, int s1) {
    constexpr int RC = GTile<KC>::RC;
    int s = s0;
    if ((s & 1) && s < s1) {   // the pair loads start at an even column
        c2 v0[RC];
        load_vec<KC>(V, s, cg, v0);
#pragma unroll
        for (int j = 0; j < RP; ++j) {
            const c2 a0 = Mb[(p0 + j) * ldm + s];
#pragma unroll
            for (int q = 0; q < RC; ++q) cfma(acc[j][q], a0, v0[q]);
        }
        ++s;
    }
#pragma unroll 2
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
#pragma unroll 4
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

// Shared memory of either sweep: Linv, two Z buffers and three [64][KC]
// vector panels (down: y_odd, r; up: r / w and the two halves of x).
template <int KC>
constexpr size_t gsmem_bytes() {
    return (size_t)(kGMT * kGLdL + 2 * kGMT * kGLdZ + 3 * kGMT * KC) * sizeof(c2);
}

// ------------------------------------------------------------------ down

// Shared memory: sLi [64][66], sZ [2][64][130], sY (y_odd) and sR (r), each
// [64][KC].  Copy groups: A(n) = Linv and y_odd of the CTA's n-th item,
// issued after the first product of item n-1; Z(n) into buffer n & 1, issued
// after the second product of item n-2.  Commit order A0 Z0 Z1 | A1 Z2 | A2
// Z3 | ..., so at the start of item n "all but the newest group" covers A(n)
// and Z(n), and before its second product "all but the newest two" covers
// Z(n).  y_even is read straight into registers before the second product.
template <int KC>
__global__ void __launch_bounds__(kGThreads, 1) k_solve_down_g32(LevelArgsT<float> a) {
    using T = GTile<KC>;
    constexpr int RC = T::RC, CG = T::CG, RG = T::RG;
    constexpr int RPA = kGMT / RG, RPB = 2 * kGMT / RG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2 *sLi = reinterpret_cast<c2 *>(smem_raw);
    c2 *sZ0 = sLi + kGMT * kGLdL;
    c2 *sY = sZ0 + 2 * kGMT * kGLdZ;
    c2 *sR = sY + kGMT * KC;

    const int m = a.m, k = a.k, tid = threadIdx.x, warp = tid >> 5;
    const int64_t mm = (int64_t)m * m, mk = (int64_t)m * k;
    const int nch = (k + KC - 1) / KC;
    const int64_t items = a.no * nch;
    const int cg = tid % CG, rg = tid / CG;
    const bool wideL = (m & 1) == 0, wideV = (k & 1) == 0;

    auto issue_a = [&](int64_t it) {
        if (it < items) {
            const int64_t t = it / nch;
            const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
            copy_tile(sLi, kGLdL, a.L + t * mm, m, m, m, wideL,
                      [&](int64_t i) { return CRS_IN(a, kDbgL, t * mm + i); });
            copy_tile(sY, KC, a.y + 2 * t * mk + c0, k, m, kw, wideV,
                      [&](int64_t i) { return CRS_IN(a, kDbgY, 2 * t * mk + c0 + i); });
        }
        cp_async_commit();
    };
    auto issue_z = [&](int64_t it, int buf) {
        if (it < items) {
            const int64_t t = it / nch;
            copy_tile(sZ0 + buf * kGMT * kGLdZ, kGLdZ, a.Z + t * 2 * mm, 2 * m, m, 2 * m, true,
                      [&](int64_t i) { return CRS_IN(a, kDbgZ, t * 2 * mm + i); });
        }
        cp_async_commit();
    };

    int64_t it = blockIdx.x;
    if (it >= items) return;
    issue_a(it);
    issue_z(it, 0);
    issue_z(it + gridDim.x, 1);
    for (int n = 0; it < items; it += gridDim.x, ++n) {
        const int64_t t = it / nch;
        const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
        const c2 *sZ = sZ0 + (n & 1) * kGMT * kGLdZ;

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
        issue_a(it + gridDim.x);
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
        c2 ye[RPB][RC];
#pragma unroll
        for (int j = 0; j < RPB; ++j) {
            const int i = rg * RPB + j - m;
#pragma unroll
            for (int q = 0; q < RC; ++q) {
                const int c = T::col(cg, q);
                const int64_t o = (2 * t + 1) * mk + (int64_t)i * k + c0 + c;
                ye[j][q] = (i >= 0 && i < m && c < kw && t < a.ne && CRS_IN(a, kDbgY, o)) ? __ldg(a.y + o)
                                                                                           : make_float2(0.f, 0.f);
            }
        }
        cp_async_wait<2>();
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
                    if (CRS_IN(a, kDbgYn, t * mk + i * k + c0 + c)) a.yn[t * mk + i * k + c0 + c] = zsub(ye[j][q], ub[j][q]);
                }
            }
        }
        __syncthreads();   // Z and r read: this Z buffer may take item n + 2
        issue_z(it + 2 * (int64_t)gridDim.x, n & 1);
    }
    cp_async_wait<0>();
}

// -------------------------------------------------------------------- up

// Shared memory: sZ [2][64][130], sLi [64][66], sR (r, then w) [64][KC], sX
// ([x_left; x_right]) [128][KC].  Copy groups: X(n) = x_left, x_right of the
// CTA's n-th item and Z(n+1) into buffer (n+1) & 1, each issued after the
// first product of item n-1; L(n) = Linv and r, issued after the second
// product of item n-1.  Commit order Z0 X0 Z1 L0 | X1 Z2 L1 | X2 Z3 L2 | ...,
// so "all but the newest two groups" covers X(n) and Z(n) at the start of
// item n and L(n) before its second product.
template <int KC>
__global__ void __launch_bounds__(kGThreads, 1) k_solve_up_g32(LevelArgsT<float> a) {
    using T = GTile<KC>;
    constexpr int RC = T::RC, CG = T::CG, RG = T::RG;
    constexpr int RP = kGMT / RG;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    c2 *sZ0 = reinterpret_cast<c2 *>(smem_raw);
    c2 *sLi = sZ0 + 2 * kGMT * kGLdZ;
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

    auto issue_z = [&](int64_t it, int buf) {
        if (it < items) {
            const int64_t t = it / nch;
            copy_tile(sZ0 + buf * kGMT * kGLdZ, kGLdZ, a.Z + t * 2 * mm, 2 * m, m, 2 * m, true,
                      [&](int64_t i) { return CRS_IN(a, kDbgZ, t * 2 * mm + i); });
        }
        cp_async_commit();
    };
    auto issue_x = [&](int64_t it) {
        if (it < items) {
            const int64_t t = it / nch;
            const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
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
        }
        cp_async_commit();
    };
    auto issue_l = [&](int64_t it) {
        if (it < items) {
            const int64_t t = it / nch;
            const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
            copy_tile(sLi, kGLdL, a.L + t * mm, m, m, m, wideL,
                      [&](int64_t i) { return CRS_IN(a, kDbgL, t * mm + i); });
            copy_tile(sR, KC, a.r + t * mk + c0, k, m, kw, wideV,
                      [&](int64_t i) { return CRS_IN(a, kDbgR, t * mk + c0 + i); });
        }
        cp_async_commit();
    };

    int64_t it = blockIdx.x;
    if (it >= items) return;
    issue_z(it, 0);
    issue_x(it);
    issue_z(it + gridDim.x, 1);
    issue_l(it);
    for (int n = 0; it < items; it += gridDim.x, ++n) {
        const int64_t t = it / nch, nxt = it + gridDim.x;
        const int c0 = (int)(it - t * nch) * KC, kw = min(KC, k - c0);
        const c2 *sZ = sZ0 + (n & 1) * kGMT * kGLdZ;

        // Z [x_left; x_right]
        cp_async_wait<2>();
        __syncthreads();
        if (t < a.ne) {
            // the even unknowns of this level are the next level's
            for (int e = tid; e < m * kw; e += kGThreads) {
                const int i = e / kw, c = e - i * kw;
                if (CRS_IN(a, kDbgX, (2 * t + 1) * mk + i * k + c0 + c))
                    a.x[(2 * t + 1) * mk + i * k + c0 + c] = sX[(m + i) * KC + c];
            }
        }
        // half h of the CTA reduces over s in [h m, (h + 1) m): P x_left or Q x_right
        constexpr int RPH = 2 * RP;
        const int h = tid / (kGThreads / 2), rgh = (tid % (kGThreads / 2)) / CG;
        c2 ah[RPH][RC];
#pragma unroll
        for (int j = 0; j < RPH; ++j)
#pragma unroll
            for (int q = 0; q < RC; ++q) ah[j][q] = make_float2(0.f, 0.f);
        gemm_rows<KC, RPH>(ah, sZ, kGLdZ, rgh * RPH, sX, cg, h * m, (h + 1) * m);
        __syncthreads();   // this Z buffer and x read: they may take items n + 2 and n + 1
        issue_x(nxt);
        issue_z(it + 2 * (int64_t)gridDim.x, n & 1);

        // w = r - P x_left - Q x_right, in place of r (each half its own
        // entries in turn, after every thread's copies of r have landed)
        cp_async_wait<2>();
        __syncthreads();
        for (int hh = 0; hh < 2; ++hh) {
            if (h == hh) {
#pragma unroll
                for (int j = 0; j < RPH; ++j) {
                    const int i = rgh * RPH + j;
#pragma unroll
                    for (int q = 0; q < RC; ++q) {
                        const int c = T::col(cg, q);
                        sR[i * KC + c] = zsub(sR[i * KC + c], ah[j][q]);
                    }
                }
            }
            __syncthreads();
        }

        // x_odd = Linv^H w (Linv^H upper triangular: a warp's rows start at
        // row warp * rows-per-warp, so its reduction starts there)
        c2 acc[RP][RC];
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
        __syncthreads();   // Linv and w read: the next item's group L may land
        issue_l(nxt);
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
    if (a.m > kGMT || a.m < 1 || a.nb != 1 || (a.kc != 8 && a.kc != 16 && a.kc != 32)) return cudaErrorInvalidValue;
    switch (a.kc) {
        case 8: return down_g32<8>(a, s);
        case 16: return down_g32<16>(a, s);
        default: return down_g32<32>(a, s);
    }
}

cudaError_t launch_solve_up_g32(const LevelArgsT<float> &a, cudaStream_t s) {
    if (a.m > kGMT || a.m < 1 || a.nb != 1 || (a.kc != 8 && a.kc != 16 && a.kc != 32)) return cudaErrorInvalidValue;
    switch (a.kc) {
        case 8: return up_g32<8>(a, s);
        case 16: return up_g32<16>(a, s);
        default: return up_g32<32>(a, s);
    }
}

}  // namespace crs
