// cr_core.cuh -- the per-level steps of classic cyclic reduction in FP64, as
// device functions that one CTA runs on one chunk of a level.
//
// One level (Sec. 2, eq. Formulas; 0-based: odd block t at position 2t, even
// block j at 2j+1, so odd t has the even blocks j = t-1 on its left and
// j = t on its right):
//   factor_chunk      per odd block: Cholesky A_2t = L L^H with the breakdown
//                     test, Z = [P | Q] = L^{-1} [B_{2t-1} | B_{2t}^H], and the
//                     Hermitian product Z^H Z (Sec. 4's rule), whose parts are
//                     Q^H Q (subtracted from the right even block), P^H P (from
//                     the left even block) and Q^H P (= -F, the next level's B).
//                     The even blocks whose two odd neighbours sit in the same
//                     chunk are finished there: V_j = (A_2j+1 - Q^H Q) - P^H P.
//   factor_fix_items  the even block on each chunk boundary: subtract the P^H P
//                     that the next chunk left in a scratch buffer.
//   solve_down_chunk  r = L^{-1} y_odd, v_j = (y_2j+1 - Q^H r) - P^H r, same
//                     chunk split, and solve_down_fix_items for the boundaries.
//   solve_up_chunk    x_odd = L^{-H}(r - P x_left - Q x_right); x_even copied.
//
// GPU mapping.  A chunk is nb consecutive odd blocks staged in shared memory.
// Each phase is a list of equal-cost work items (a matrix entry, a column of
// a triangular solve) spread over all threads of the CTA; items of different
// cost (pivots, real diagonal entries) get warps of their own.  On GB300 the
// FP64 pipe (2 DFMA/clk/SM) bounds this path and one warp per SM
// sub-partition with a dependent chain already keeps it ~90% busy, so lane
// utilisation and FP64 instruction count matter most, occupancy little.
// The level kernels run one chunk per CTA; the batched kernel runs all chunks
// of all levels of one system in one CTA.
#pragma once
#include <type_traits>

#include "cr_device.cuh"
#include "cr_tc.cuh"

__host__ __device__ inline int64_t crs_num_ctas(int64_t no, int nb) { return (no + nb - 1) / nb; }

namespace crs {

// Packed lower-triangular storage in shared memory: entry (r, c), r >= c.
__device__ __forceinline__ int tri(int r, int c) { return r * (r + 1) / 2 + c; }
template <int MT> struct Tri { static constexpr int n = MT * (MT + 1) / 2; };

// --------------------------------------------------------------- helpers

// z := L^{-1} z for one column z (shared memory, stride ld); L packed lower.
template <int MT, class R, class C>
__device__ __forceinline__ void trsv_lower_col(const C *Lb, const R *ivb, C *col, int ld, int m) {
    if constexpr (MT <= 16) {
        C z[MT];
#pragma unroll
        for (int r = 0; r < MT; ++r)
            if (r < m) z[r] = col[r * ld];
#pragma unroll
        for (int r = 0; r < MT; ++r) {
            if (r < m) {
                C acc = z[r];
#pragma unroll
                for (int s = 0; s < r; ++s) zmsub(acc, Lb[tri(r, s)], z[s]);
                z[r] = zscale(acc, ivb[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < MT; ++r)
            if (r < m) col[r * ld] = z[r];
    } else {
        for (int r = 0; r < m; ++r) {
            C acc = col[r * ld];
            for (int s = 0; s < r; ++s) zmsub(acc, Lb[tri(r, s)], col[s * ld]);
            col[r * ld] = zscale(acc, ivb[r]);
        }
    }
}

// z := L^{-H} z for one column z (shared memory, stride ld); L packed lower.
// Row r subtracts the terms of rows s = m-1 down to r+1, the order in which
// trsv_lower_h_wide produces them.
template <int MT, class R, class C>
__device__ __forceinline__ void trsv_lower_h_col(const C *Lb, const R *ivb, C *col, int ld, int m) {
    if constexpr (MT <= 16) {
        C z[MT];
#pragma unroll
        for (int r = 0; r < MT; ++r)
            if (r < m) z[r] = col[r * ld];
#pragma unroll
        for (int r = MT - 1; r >= 0; --r) {
            if (r < m) {
                C acc = z[r];
#pragma unroll
                for (int s = MT - 1; s > r; --s)
                    if (s < m) zmsub_ca(acc, Lb[tri(s, r)], z[s]);
                z[r] = zscale(acc, ivb[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < MT; ++r)
            if (r < m) col[r * ld] = z[r];
    } else {
        for (int r = m - 1; r >= 0; --r) {
            C acc = col[r * ld];
            for (int s = m - 1; s > r; --s) zmsub_ca(acc, Lb[tri(s, r)], col[s * ld]);
            col[r * ld] = zscale(acc, ivb[r]);
        }
    }
}

// Chunks with few columns to solve (the coarse levels, one or two odd blocks
// per CTA): a column per thread leaves most of the CTA idle while one warp
// runs a dependent chain of m(m-1)/2 complex FMAs per column, and on GB300 a
// warp's FP64 instruction holds its sub-partition's FP64 pipe for about 64
// cycles (2 DFMA per clock per SM), so that chain takes ~15 us at m = 16.
// The wide forms below take the same operations in the same order (results
// bit-identical to the column-per-thread forms) but spread each step over
// (block, row, column) items: row s is final, then every row below it is
// updated in parallel, and the next row is scaled by the item that finishes
// it, so a step costs one barrier.

// Z := L^{-1} Z for columns c < ncols of blocks b < nbh (column (b, c) at
// base + b * bstride + c, row stride ld); skip(b, c) marks columns that stay
// zero.  Same operations and order as trsv_lower_col.  Ends with
// __syncthreads().
template <int MT, class R, class C, class Skip>
__device__ __forceinline__ void trsv_lower_wide(const C *sL, const R *sInv, C *base, int bstride, int ld, int nbh,
                                                int ncols, int m, Skip skip) {
    constexpr int TRI = Tri<MT>::n;
    const int NT = blockDim.x, tid = threadIdx.x, nc = nbh * ncols;
    for (int e = tid; e < nc; e += NT) {
        const int b = e / ncols, c = e - b * ncols;
        if (skip(b, c)) continue;
        C *p = base + b * bstride + c;
        *p = zscale(*p, sInv[b * MT]);
    }
    __syncthreads();
    for (int s = 0; s + 1 < m; ++s) {
        const int nr = m - 1 - s, per_b = nr * ncols;
        for (int e = tid; e < nbh * per_b; e += NT) {
            const int b = e / per_b, rem = e - b * per_b, r = s + 1 + rem / ncols, c = rem % ncols;
            if (skip(b, c)) continue;
            C *col = base + b * bstride + c;
            C acc = col[r * ld];
            zmsub(acc, sL[b * TRI + tri(r, s)], col[s * ld]);
            if (r == s + 1) acc = zscale(acc, sInv[b * MT + r]);
            col[r * ld] = acc;
        }
        __syncthreads();
    }
}

// Z := L^{-H} Z for columns c < ncols of blocks b < nbh (layout as in
// trsv_lower_wide).  Same operations and order as trsv_lower_h_col.  Ends
// with __syncthreads().
template <int MT, class R, class C>
__device__ __forceinline__ void trsv_lower_h_wide(const C *sL, const R *sInv, C *base, int bstride, int ld, int nbh,
                                                  int ncols, int m) {
    constexpr int TRI = Tri<MT>::n;
    const int NT = blockDim.x, tid = threadIdx.x, nc = nbh * ncols;
    for (int e = tid; e < nc; e += NT) {
        const int b = e / ncols, c = e - b * ncols;
        C *p = base + b * bstride + c + (m - 1) * ld;
        *p = zscale(*p, sInv[b * MT + m - 1]);
    }
    __syncthreads();
    for (int s = m - 1; s >= 1; --s) {
        const int per_b = s * ncols;   // rows 0 .. s-1
        for (int e = tid; e < nbh * per_b; e += NT) {
            const int b = e / per_b, rem = e - b * per_b, r = rem / ncols, c = rem % ncols;
            C *col = base + b * bstride + c;
            C acc = col[r * ld];
            zmsub_ca(acc, sL[b * TRI + tri(s, r)], col[s * ld]);
            if (r == s - 1) acc = zscale(acc, sInv[b * MT + r]);
            col[r * ld] = acc;
        }
        __syncthreads();
    }
}

// Right-looking Cholesky A_b = L_b L_b^H of the blocks b < nbh of a chunk
// (packed lower in sL, 1 / diag(L) to sInv) with the breakdown test of
// factor_chunk: the same operations in the same order as its left-looking
// column steps (entry (r, q) subtracts L_rs conj(L_qs) for s = 0 .. q-1 in
// turn, the pivot d = A_qq - sum |L_qs|^2 by two real FMAs per term), so L is
// bit-identical.  Per column: scale the column below the pivot, then update
// the trailing triangle in parallel; the item that finishes the next
// diagonal entry takes its pivot.  Ends with __syncthreads().
template <int MT, class R, class C>
__device__ __forceinline__ void chol_lower_wide(const LevelArgsT<R> &a, int64_t t0, C *sL, R *sInv, int nbh, int m) {
    constexpr int TRI = Tri<MT>::n;
    const int NT = blockDim.x, tid = threadIdx.x;
    auto pivot = [&](int b, int c, R d) {
        if (!(d > R(0))) report_fail(a.status, a.level, report_index(a, 2 * (t0 + b)));
        const R iv = rsq(d);
        sInv[b * MT + c] = iv;
        sL[b * TRI + tri(c, c)] = zmk(d * iv, R(0));
    };
    for (int b = tid; b < nbh; b += NT) pivot(b, 0, sL[b * TRI].x);
    __syncthreads();
    for (int c = 0; c + 1 < m; ++c) {
        const int below = m - 1 - c, ntr = below * (below + 1) / 2;
        for (int e = tid; e < nbh * below; e += NT) {
            const int b = e / below, r = c + 1 + (e - b * below);
            C *p = sL + b * TRI + tri(r, c);
            *p = zscale(*p, sInv[b * MT + c]);
        }
        __syncthreads();
        for (int e = tid; e < nbh * ntr; e += NT) {
            const int b = e / ntr, f = e - b * ntr, rr = tri_row(f), qq = f - rr * (rr + 1) / 2;
            const int r = c + 1 + rr, q = c + 1 + qq;
            C *Lb = sL + b * TRI;
            const C lr = Lb[tri(r, c)];
            if (r == q) {
                R d = Lb[tri(r, r)].x;
                d = fmx(-lr.x, lr.x, d);
                d = fmx(-lr.y, lr.y, d);
                if (r == c + 1) pivot(b, r, d);
                else Lb[tri(r, r)].x = d;
            } else {
                C u = Lb[tri(r, q)];
                zmsub_cb(u, lr, Lb[tri(q, c)]);
                Lb[tri(r, q)] = u;
            }
        }
        __syncthreads();
    }
}

// Blocked forward substitution Z := L^{-1} Z for every column of every block
// of a chunk, run by the whole CTA (used for MT >= 32, where a column-by-
// column substitution would be one long dependent chain per thread).  Rows
// are taken in blocks of 16: the diagonal block is solved per column (a
// chain of <= 16 rows), then the rows below are updated in parallel, one
// item per (block, row, column).  Column (b, col) starts at
// base + b * bstride + col, with row stride ld.  With kUnit2, a second set of
// ncols2 columns at base2 + b * bstride2 + j (row stride ld2) is solved in the
// same passes; column j of it must start as the unit vector e_j, so its rows
// above j are zero and stay zero and the items that would only add zeros
// are skipped (ncols2 = m gives L^{-1}).  Ends with __syncthreads().
template <int MT, class R, class C, bool kUnit2 = false>
__device__ __forceinline__ void trsm_lower_cta(const C *sL, const R *sInv, C *base, int bstride, int ld, int nbh,
                                               int ncols, int m, C *base2 = nullptr, int bstride2 = 0, int ld2 = 0,
                                               int ncols2 = 0) {
    constexpr int TRI = Tri<MT>::n, BS = 16;
    const int NT = blockDim.x, tid = threadIdx.x;
    const int ntot = kUnit2 ? ncols + ncols2 : ncols;
    for (int rb = 0; rb < m; rb += BS) {
        const int re = min(rb + BS, m);
        const int nbr = re - rb;
        for (int e = tid; e < nbh * ntot; e += NT) {
            const int b = e / ntot, col = e - b * ntot;
            const C *Lb = sL + b * TRI;
            const R *ivb = sInv + b * MT;
            C *z = base + b * bstride + col;
            int ld_ = ld;
            if constexpr (kUnit2) {
                if (col >= ncols) {
                    const int j = col - ncols;
                    if (j >= re) continue;   // rows rb .. re-1 of e_j are zero
                    z = base2 + b * bstride2 + j;
                    ld_ = ld2;
                }
            }
            if constexpr (sizeof(R) == 4) {
                // FP32 (latency-bound): the column's rows rb .. re-1 in
                // registers, so the chain waits on FMAs, not on shared memory
                C zr[BS];
#pragma unroll
                for (int i = 0; i < BS; ++i)
                    if (i < nbr) zr[i] = z[(rb + i) * ld_];
#pragma unroll
                for (int i = 0; i < BS; ++i) {
                    if (i < nbr) {
                        const C *Lr = Lb + tri(rb + i, rb);
                        C acc = zr[i];
#pragma unroll
                        for (int j = 0; j < i; ++j) zmsub(acc, Lr[j], zr[j]);
                        zr[i] = zscale(acc, ivb[rb + i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < BS; ++i)
                    if (i < nbr) z[(rb + i) * ld_] = zr[i];
            } else {
                for (int r = rb; r < re; ++r) {
                    C acc = z[r * ld_];
                    for (int s = rb; s < r; ++s) zmsub(acc, Lb[tri(r, s)], z[s * ld_]);
                    z[r * ld_] = zscale(acc, ivb[r]);
                }
            }
        }
        __syncthreads();
        if (re < m) {
            const int nr = m - re, per = nr * ntot;
            for (int e = tid; e < nbh * per; e += NT) {
                const int b = e / per, rem = e - b * per, r = re + rem / ntot, col = rem - (r - re) * ntot;
                const C *Lr = sL + b * TRI + tri(r, 0);
                C *z = base + b * bstride + col;
                int ld_ = ld;
                if constexpr (kUnit2) {
                    if (col >= ncols) {
                        const int j = col - ncols;
                        if (j >= re) continue;   // rows rb .. re-1 of this column are zero
                        z = base2 + b * bstride2 + j;
                        ld_ = ld2;
                    }
                }
                C acc = z[r * ld_];
#pragma unroll 4
                for (int s = rb; s < re; ++s) zmsub(acc, Lr[s], z[s * ld_]);
                z[r * ld_] = acc;
            }
            __syncthreads();
        }
    }
}

// Blocked backward substitution Z := L^{-H} Z, the mirror of trsm_lower_cta:
// row blocks from the bottom, the diagonal block per column, then the rows
// above updated in parallel.  Ends with __syncthreads().
template <int MT, class R, class C>
__device__ __forceinline__ void trsm_lower_h_cta(const C *sL, const R *sInv, C *base, int bstride, int ld, int nbh,
                                                 int ncols, int m) {
    constexpr int TRI = Tri<MT>::n, BS = 16;
    const int NT = blockDim.x, tid = threadIdx.x;
    for (int re = m; re > 0; re -= BS) {
        const int rb = max(re - BS, 0);
        const int nbr = re - rb;
        for (int e = tid; e < nbh * ncols; e += NT) {
            const int b = e / ncols, col = e - b * ncols;
            const C *Lb = sL + b * TRI;
            const R *ivb = sInv + b * MT;
            C *z = base + b * bstride + col;
            if constexpr (sizeof(R) == 4) {
                C zr[BS];
#pragma unroll
                for (int i = 0; i < BS; ++i)
                    if (i < nbr) zr[i] = z[(rb + i) * ld];
#pragma unroll
                for (int i = BS - 1; i >= 0; --i) {
                    if (i < nbr) {
                        C acc = zr[i];
#pragma unroll
                        for (int j = i + 1; j < BS; ++j)
                            if (j < nbr) zmsub_ca(acc, Lb[tri(rb + j, rb + i)], zr[j]);
                        zr[i] = zscale(acc, ivb[rb + i]);
                    }
                }
#pragma unroll
                for (int i = 0; i < BS; ++i)
                    if (i < nbr) z[(rb + i) * ld] = zr[i];
            } else {
                for (int r = re - 1; r >= rb; --r) {
                    C acc = z[r * ld];
                    for (int s = r + 1; s < re; ++s) zmsub_ca(acc, Lb[tri(s, r)], z[s * ld]);
                    z[r * ld] = zscale(acc, ivb[r]);
                }
            }
        }
        __syncthreads();
        if (rb > 0) {
            const int per = rb * ncols;
            for (int e = tid; e < nbh * per; e += NT) {
                const int b = e / per, rem = e - b * per, r = rem / ncols, col = rem - r * ncols;
                const C *Lb = sL + b * TRI;
                C *z = base + b * bstride + col;
                C acc = z[r * ld];
#pragma unroll 4
                for (int s = rb; s < re; ++s) zmsub_ca(acc, Lb[tri(s, r)], z[s * ld]);
                z[r * ld] = acc;
            }
            __syncthreads();
        }
    }
}

}  // namespace crs
#include "cr_factor32.cuh"   // blocked FP32 factor of class MT = 64 (uses tri, trsm helpers above)
namespace crs {

// ---------------------------------------------- FP32 Schur products (tcgen05)

// Shared memory of the tensor-core Schur product: 1 KB for two mbarriers and
// the TMEM address, then two operand buffers (double buffering over the
// K-stages), each holding the three TF32 pieces of one stage of X (2MT rows
// x kTcKS K-columns of 32-bit elements).
constexpr int kTcKS = 16;
__host__ __device__ constexpr size_t tc_stage_bytes(int mt) {
    return 1024 + 2 * 3 * (size_t)(2 * mt) * kTcKS * 4;
}

// Lower triangle of Z^H Z for one block on the tensor cores (FP32 levels of
// the mixed form, MT = 64).  With X = [Re Z; Im Z] (real, rows s' = 0..2m-1,
// column p = column of Z), Re(Z^H Z) = X^T X and
// Im(Z^H Z) = (Re Z)^T (Im Z) - (Im Z)^T (Re Z): three real products with
// M = N = 2MT = 128 into three TMEM accumulators (the imaginary part as the
// difference of the last two, formed when it is read).  X is stored once per
// K-stage: rows s0..s0+7 of Re Z as K-columns 0..7 and the same rows of Im Z
// as K-columns 8..15, so X^T X takes both halves and the cross products one
// half each as A and the other as B.  Every FP32 operand is split exactly
// into three TF32 pieces x = x1 + x2 + x3 (11 significant bits each), and
// the six products x1 y1, x1 y2, x2 y1, x1 y3, x2 y2, x3 y1 (smallest first)
// are accumulated in FP32: the dropped terms are below 2^-33 of the product,
// so the result has the accuracy of FP32 arithmetic, which the iterative
// refinement needs.  The stages alternate between two operand buffers: while
// the MMAs of one stage run, the threads split the next stage into the other
// buffer (an mbarrier per buffer, completed by the MMAs' commit, says when a
// buffer may be refilled; uses0 / uses1 count their commits).  All eight warps
// then read the accumulators (row p = lane of TMEM, two warps per lane group,
// column chunks split between them) and route the entries: P^H P (q <= p < m)
// to sW, Q^H Q (m <= q <= p) subtracted from sV, and the next level's B =
// -Q^H P from the upper triangle (p < m <= q), where consecutive lanes hold
// consecutive entries of a row of B.
// Returns false if a wait gave up.
template <int MT>
__device__ __forceinline__ bool herk_tc_f32(const LevelArgsT<float> &a, int64_t t, const float2 *Zb, float2 *sWb, float2 *sVb,
                            unsigned char *stage, uint32_t &uses0, uint32_t &uses1, uint32_t &stage_count) {
    constexpr int M = 2 * MT, KS = kTcKS, HS = KS / 2;
    constexpr int PIECE = M * KS * 4;
    const int m = a.m, m2 = 2 * m, NT = blockDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int mm = m * m;
    uint64_t *mbar = reinterpret_cast<uint64_t *>(stage);
    const uint32_t tmem = *reinterpret_cast<uint32_t *>(stage + 16);
    unsigned char *ops = stage + 1024;
    constexpr uint32_t idesc = idesc_tf32(M, M);
    bool ok = true;
    auto split3 = [](float v, uint32_t &p1, uint32_t &p2, uint32_t &p3) {
        p1 = cvt_tf32(v);
        const float r1 = v - __uint_as_float(p1);
        p2 = cvt_tf32(r1);
        p3 = cvt_tf32(r1 - __uint_as_float(p2));
    };
    const int nst = (m + HS - 1) / HS;
    for (int ks = 0; ks < nst; ++ks) {
        const int buf = (int)(stage_count & 1u);
        const uint32_t ub = buf ? uses1 : uses0;
        // the buffer's previous MMAs must have read it; a wait that gives up
        // (in any thread) ends the product for the whole CTA
        const bool got = ub == 0 || mbar_wait(smem_u32(&mbar[buf]), (ub - 1) & 1u, 1 << 24);
        if (__syncthreads_or(!got)) {
            ok = false;
            break;
        }
        unsigned char *B0 = ops + buf * 3 * PIECE;
        // item e: K-column kk = 4 kh + (e & 3) of the top half (Re Z row
        // s = ks*HS + kk) and kk + HS of the bottom half (Im Z of the same
        // row), operand row i = 8 ig + ((e >> 2) & 7); consecutive lanes
        // write consecutive words of a core matrix
        for (int e = tid; e < M * HS; e += NT) {
            const int kk = ((e >> 5) & 1) * 4 + (e & 3), i = (e >> 6) * 8 + ((e >> 2) & 7);
            const int sr = ks * HS + kk;
            float2 z = make_float2(0.f, 0.f);
            if (sr < m && i < m2) z = Zb[sr * 2 * MT + i];
            uint32_t p[3];
            split3(z.x, p[0], p[1], p[2]);
            const int ot = kmaj_off(i, kk, KS), ob = kmaj_off(i, kk + HS, KS);
#pragma unroll
            for (int c = 0; c < 3; ++c) *reinterpret_cast<uint32_t *>(B0 + c * PIECE + ot) = p[c];
            split3(z.y, p[0], p[1], p[2]);
#pragma unroll
            for (int c = 0; c < 3; ++c) *reinterpret_cast<uint32_t *>(B0 + c * PIECE + ob) = p[c];
        }
        fence_async_smem();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        if (tid == 0) {
            // (A piece, B piece), smallest terms first
            const int pa[6] = {2, 1, 0, 1, 0, 0}, pb[6] = {0, 1, 2, 0, 1, 0};
            const uint32_t b0 = smem_u32(B0);
#pragma unroll
            for (int pass = 0; pass < 6; ++pass) {
                const uint32_t ab = b0 + pa[pass] * PIECE, bb = b0 + pb[pass] * PIECE;
                const uint64_t at = umma_desc(ab, 128, (KS / 4) * 128), abot = umma_desc(ab + 256, 128, (KS / 4) * 128);
                const uint64_t bt = umma_desc(bb, 128, (KS / 4) * 128), bbot = umma_desc(bb + 256, 128, (KS / 4) * 128);
                const uint32_t first = (ks == 0 && pass == 0) ? 0u : 1u;
                mma_tf32(tmem, at, bt, idesc, first);                 // Re: X^T X, top half
                mma_tf32(tmem, abot, bbot, idesc, 1u);                //     and bottom half
                mma_tf32(tmem + M, at, bbot, idesc, first);           // (Re Z)^T (Im Z)
                mma_tf32(tmem + 2 * M, abot, bt, idesc, first);       // (Im Z)^T (Re Z)
            }
            tc_commit(smem_u32(&mbar[buf]));
        }
        if (buf) ++uses1;
        else ++uses0;
        ++stage_count;
    }
    // all MMAs of this block: the last commit tracks every earlier one
    if (ok && stage_count > 0) {
        const int lb = (int)((stage_count - 1) & 1u);
        const bool got = mbar_wait(smem_u32(&mbar[lb]), ((lb ? uses1 : uses0) - 1) & 1u, 1 << 24);
        if (__syncthreads_or(!got)) ok = false;
    }
    tc_fence_after();
    // Epilogue by all 8 warps: warp w reads TMEM lanes 32 (w % 4) .. +31 (rows
    // p) and the column chunks c of parity w / 4.  Row p < m gives P^H P (q <= p,
    // q < m) and, from the upper triangle, the next level's B: for q in
    // [m, 2m), B_next[q - m][p] = -(Q^H P)[q - m][p] = -conj(Z^H Z)[p][q], so that
    // consecutive lanes write consecutive entries; row p >= m gives Q^H Q
    // (m <= q <= p).
    if (warp < 8) {
        const int g = warp & 3, h = warp >> 2, p = g * 32 + lane;
        const bool hasL = t >= 1, hasR = 2 * t + 1 < a.Nl;
        const int rlo = g * 32, rhi = g * 32 + 31;
        for (int c = h; c < M / 32; c += 2) {
            const int clo = c * 32, chi = c * 32 + 31;
            const bool needP = rlo < m && clo < m && clo <= rhi;
            const bool needB = rlo < m && chi >= m && clo < m2;
            const bool needQ = rhi >= m && rlo < m2 && chi >= m && clo <= rhi;
            if (!(needP || needB || needQ)) continue;   // the same in every lane of the warp
            uint32_t vr[32], v1[32], v2[32];
            const uint32_t lanes = (uint32_t)(g * 32) << 16;
            tmem_ld32(tmem + lanes + (uint32_t)clo, vr);
            tmem_ld32(tmem + lanes + (uint32_t)(M + clo), v1);
            tmem_ld32(tmem + lanes + (uint32_t)(2 * M + clo), v2);
            if (!ok || p >= m2) continue;
#pragma unroll
            for (int j = 0; j < 32; ++j) {
                const int q = clo + j;
                if (q >= m2) continue;
                const float dr = __uint_as_float(vr[j]);
                const float di = (q == p) ? 0.f : __uint_as_float(v1[j]) - __uint_as_float(v2[j]);
                if (p < m) {
                    if (q <= p) {
                        if (hasL) sWb[tri(p, q)] = make_float2(dr, di);
                    } else if (q >= m && hasL && hasR && CRS_IN(a, kDbgBn, (t - 1) * mm + (q - m) * m + p)) {
                        a.Bn[(t - 1) * mm + (q - m) * m + p] = make_float2(-dr, di);
                    }
                } else if (q >= m && q <= p && hasR) {
                    float2 &v = sVb[tri(p - m, q - m)];
                    v.x -= dr;
                    v.y -= di;
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return ok;
}

// ------------------------------------------------------------ factor: odd

// Entry f of the lower triangle of the boundary block of boundary c.  With
// kL2 the two halves are read through L2 (one of them was written by another
// CTA of the same launch).
template <class R, bool kL2 = false>
__device__ __forceinline__ void factor_fix_entry(const LevelArgsT<R> &a, int64_t c, int f) {
    using C = cplx_t<R>;
    const int m = a.m, mm = m * m;
    const int p = tri_row(f), q = f - p * (p + 1) / 2;
    const int64_t j = c * a.nb - 1;
    if (!CRS_IN(a, kDbgAn, j * mm + p * m + q) || !CRS_IN(a, kDbgAn, j * mm + q * m + p) ||
        !CRS_IN(a, kDbgWbd, c * mm + p * m + q))
        return;
    const C *pa = a.An + j * mm + p * m + q, *pw = a.Wbd + c * mm + p * m + q;
    C v = kL2 ? zsub(__ldcg(pa), __ldcg(pw)) : zsub(*pa, *pw);
    if (p == q) v.y = R(0);
    a.An[j * mm + p * m + q] = v;
    if (p != q) a.An[j * mm + q * m + p] = zconj(v);
}

// Completion of the chunk-boundary even blocks inside the odd-block kernels
// (a.bd_count set).  The even block on the boundary between chunks c-1 and
// c gets one half from each of the two CTAs: chunk c-1 leaves it without
// its right neighbour's term, chunk c leaves that term (in Wbd or cbd).
// Each CTA, once its stores are out, counts itself in at its boundaries; the
// second to arrive completes the block with the fix-up kernels' subtraction
// (same result) and resets the counter for the next launch.  No CTA waits
// for another.  Called by every thread of the CTA; returns bit 0 when this
// CTA completes its left boundary (c = chunk), bit 1 its right one (chunk + 1).
__device__ __forceinline__ int bd_arrive(unsigned *cnt, int64_t chunk, int64_t ncta) {
    __threadfence();   // this thread's stores, before the CTA's arrival
    __syncthreads();
    int second = 0;
    if (threadIdx.x == 0) {
        if (chunk >= 1 && atomicAdd(cnt + chunk, 1u) == 1u) {
            cnt[chunk] = 0u;
            second |= 1;
        }
        if (chunk + 1 < ncta && atomicAdd(cnt + chunk + 1, 1u) == 1u) {
            cnt[chunk + 1] = 0u;
            second |= 2;
        }
        __threadfence();   // the other CTA's stores, before this CTA reads them
    }
    const int left = __syncthreads_or(second & 1), right = __syncthreads_or(second & 2);
    return (left ? 1 : 0) | (right ? 2 : 0);
}

// One chunk of nb odd blocks (chunk index `chunk`) of a factor level, run by
// the whole CTA.  Uses the CTA's shared memory from smem_raw.
template <int MT, class R, bool kWide = false>
__device__ __forceinline__ void factor_chunk(const LevelArgsT<R> &a, int64_t chunk, unsigned char *smem_raw) {
    using C = cplx_t<R>;
    constexpr int LDZ = 2 * MT, TRI = Tri<MT>::n;
    const int m = a.m, nb = a.nb, NT = blockDim.x, tid = threadIdx.x;
    const int mm = m * m, m2 = 2 * m;
    const int64_t t0 = chunk * nb;
    const int nbh = (int)min((int64_t)nb, a.no - t0);
    C *sL = reinterpret_cast<C *>(smem_raw);                        // [nb][TRI] L, later P^H P
    C *sV = sL + (size_t)nb * TRI;                                    // [nb][TRI] even block t0+b
    C *sZ = sV + (size_t)nb * TRI;                                    // [nb][MT][2MT] [P | Q]
    R *sInv = reinterpret_cast<R *>(sZ + (size_t)nb * MT * LDZ);  // [nb][MT]
    // FP32 levels of class MT = 64 (the mixed form): the factorisation runs by
    // 16 x 16 blocks (cr_factor32.cuh) and also forms L^{-1}, which is kept in
    // place of L for the product form of the solves (cr_solve32.cu);
    // [nb][MT][kF32LdE] after the tensor-core operand stages, zeroed here
    constexpr bool kLinv = std::is_same<R, float>::value && MT == 64;
    C *sLi = nullptr;
    if constexpr (kLinv) {
        unsigned char *st = reinterpret_cast<unsigned char *>(
            (reinterpret_cast<uintptr_t>(sInv + (size_t)nb * MT) + 1023) & ~(uintptr_t)1023);
        sLi = reinterpret_cast<C *>(st + tc_stage_bytes(MT));
        for (int e = tid; e < nbh * MT * kF32LdE; e += NT) sLi[e] = zmk(R(0), R(0));
    }

    // stage the lower triangles of A_2t and A_2t+1, B_{2t-1} (P part) and
    // B_{2t}^H (Q part)
    if constexpr (kLinv) {
        stage_f32_64<MT>(a, t0, nbh, sL, sV, sZ);
    } else if constexpr (MT >= 32 && sizeof(R) == 4) {
        // FP32 large tiles (one or two CTAs per SM, latency-bound): the loads
        // of U iterations go out together
        // (into registers) before any store, so their latencies overlap
        constexpr int U = 8;
        const int n = nbh * mm;
        for (int e0 = tid; e0 < n; e0 += U * NT) {
            C va[U], vv[U], vp[U], vq[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * NT;
                va[u] = vv[u] = vp[u] = vq[u] = zmk(R(0), R(0));
                if (e < n) {
                    const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
                    const int64_t t = t0 + b, pos = 2 * t;
                    if (r >= c) {
                        if (CRS_IN(a, kDbgA, pos * mm + rem)) va[u] = __ldg(a.A + pos * mm + rem);
                        if (t < a.ne && CRS_IN(a, kDbgA, (pos + 1) * mm + rem)) vv[u] = __ldg(a.A + (pos + 1) * mm + rem);
                    }
                    if (pos >= 1 && CRS_IN(a, kDbgB, (pos - 1) * mm + rem)) vp[u] = __ldg(a.B + (pos - 1) * mm + rem);
                    if (pos + 1 < a.Nl && CRS_IN(a, kDbgB, pos * mm + rem)) vq[u] = __ldg(a.B + pos * mm + rem);
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int e = e0 + u * NT;
                if (e < n) {
                    const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
                    if (r >= c) {
                        sL[b * TRI + tri(r, c)] = va[u];
                        if (t0 + b < a.ne) {
                            C v = vv[u];
                            if (r == c) v.y = R(0);
                            sV[b * TRI + tri(r, c)] = v;
                        }
                    }
                    sZ[(b * MT + r) * LDZ + c] = vp[u];
                    sZ[(b * MT + c) * LDZ + m + r] = zconj(vq[u]);
                }
            }
        }
    } else {
        for (int e = tid; e < nbh * mm; e += NT) {
            const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
            const int64_t t = t0 + b, pos = 2 * t;
            if (r >= c) {
                sL[b * TRI + tri(r, c)] = CRS_IN(a, kDbgA, pos * mm + rem) ? a.A[pos * mm + rem] : zmk(R(0), R(0));
                if (t < a.ne) {
                    C v = CRS_IN(a, kDbgA, (pos + 1) * mm + rem) ? a.A[(pos + 1) * mm + rem] : zmk(R(0), R(0));
                    if (r == c) v.y = R(0);
                    sV[b * TRI + tri(r, c)] = v;
                }
            }
            sZ[(b * MT + r) * LDZ + c] =
                (pos >= 1 && CRS_IN(a, kDbgB, (pos - 1) * mm + rem)) ? a.B[(pos - 1) * mm + rem] : zmk(R(0), R(0));
            sZ[(b * MT + c) * LDZ + m + r] =
                (pos + 1 < a.Nl && CRS_IN(a, kDbgB, pos * mm + rem)) ? zconj(a.B[pos * mm + rem]) : zmk(R(0), R(0));
        }
    }
    __syncthreads();

    if constexpr (kLinv) {
        for (int b = 0; b < nbh; ++b)
            chol_inv_z_f32<MT>(a, report_index(a, 2 * (t0 + b)), sL + b * TRI, sInv + b * MT, sLi + b * MT * kF32LdE,
                               sZ + b * MT * LDZ);
    } else {
        if constexpr (MT < 32 && kWide) {
            chol_lower_wide<MT, R, C>(a, t0, sL, sInv, nbh, m);
            // zero columns stay zero, as below
            trsv_lower_wide<MT, R, C>(sL, sInv, sZ, MT * LDZ, LDZ, nbh, m2, m, [&](int b, int col) {
                const int64_t pos = 2 * (t0 + b);
                return col < m ? (pos == 0) : (pos + 1 >= a.Nl);
            });
        } else {
            // Cholesky by panels of PW columns (one panel of m columns when MT < 32).
            // Inside a panel, left-looking by columns: pass 1 of column c computes the
            // pivots (one item per block, in warps of their own so that the sqrt path
            // does not diverge from the off-diagonal path) and the unscaled entries
            // below the pivot, summing only over the panel's earlier columns; pass 2
            // scales them by 1 / pivot.  After a panel, the trailing lower triangle is
            // updated in parallel (one item per entry), so the dependent chains of the
            // column steps stay shorter than PW.
            const int dpad = (nbh + 31) & ~31;
            const int PW = (MT >= 32) ? 16 : m;
            for (int kb = 0; kb < m; kb += PW) {
                const int ke = min(kb + PW, m);
                for (int c = kb; c < ke; ++c) {
                    const int below = m - c - 1;
                    for (int e = tid; e < dpad + nbh * below; e += NT) {
                        if (e < nbh) {
                            const int b = e;
                            C *Lb = sL + b * TRI;
                            R d = Lb[tri(c, c)].x;
                            if constexpr (MT >= 32 && sizeof(R) == 4) {
                                // fixed trip count: the loads are issued ahead of the FMA chain
                                const C *Lc = Lb + tri(c, kb);
        #pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    if (kb + j < c) {
                                        const C l = Lc[j];
                                        d = fmx(-l.x, l.x, d);
                                        d = fmx(-l.y, l.y, d);
                                    }
                            } else {
                                for (int s = kb; s < c; ++s) {
                                    const C l = Lb[tri(c, s)];
                                    d = fmx(-l.x, l.x, d);
                                    d = fmx(-l.y, l.y, d);
                                }
                            }
                            if (!(d > R(0))) report_fail(a.status, a.level, report_index(a, 2 * (t0 + b)));
                            const R iv = rsq(d);
                            sInv[b * MT + c] = iv;
                            Lb[tri(c, c)] = zmk(d * iv, R(0));
                        } else if (e >= dpad) {
                            const int e2 = e - dpad, b = e2 / below, r = c + 1 + (e2 - b * below);
                            C *Lb = sL + b * TRI;
                            C u = Lb[tri(r, c)];
                            if constexpr (MT >= 32 && sizeof(R) == 4) {
                                const C *Lr = Lb + tri(r, kb), *Lc = Lb + tri(c, kb);
        #pragma unroll
                                for (int j = 0; j < 16; ++j)
                                    if (kb + j < c) zmsub_cb(u, Lr[j], Lc[j]);
                            } else {
                                for (int s = kb; s < c; ++s) zmsub_cb(u, Lb[tri(r, s)], Lb[tri(c, s)]);
                            }
                            Lb[tri(r, c)] = u;
                        }
                    }
                    __syncthreads();
                    for (int e = tid; e < nbh * below; e += NT) {
                        const int b = e / below, r = c + 1 + (e - b * below);
                        C *p = sL + b * TRI + tri(r, c);
                        *p = zscale(*p, sInv[b * MT + c]);
                    }
                    __syncthreads();
                }
                if (ke < m) {
                    // A[r][q] -= sum_{s in panel} L[r][s] conj(L[q][s]) for ke <= q <= r < m
                    const int nr = m - ke, ntr = nr * (nr + 1) / 2;
                    for (int e = tid; e < nbh * ntr; e += NT) {
                        const int b = e / ntr, f = e - b * ntr, rr = tri_row(f), qq = f - rr * (rr + 1) / 2;
                        const int r = ke + rr, q = ke + qq;
                        C *Lb = sL + b * TRI;
                        C u = Lb[tri(r, q)];
                        if constexpr (sizeof(R) == 4) {
                            const C *Lr = Lb + tri(r, kb), *Lq = Lb + tri(q, kb);
        #pragma unroll
                            for (int j = 0; j < 16; ++j)
                                if (kb + j < ke) zmsub_cb(u, Lr[j], Lq[j]);
                        } else {
                            for (int s = kb; s < ke; ++s) zmsub_cb(u, Lb[tri(r, s)], Lb[tri(q, s)]);
                        }
                        Lb[tri(r, q)] = u;
                    }
                    __syncthreads();
                }
            }

            // Z := L^{-1} Z, one item per (block, column); zero columns stay zero
            if constexpr (MT >= 32) {
                trsm_lower_cta<MT, R, C>(sL, sInv, sZ, MT * LDZ, LDZ, nbh, m2, m);
            } else {
                for (int e = tid; e < nbh * m2; e += NT) {
                    const int b = e / m2, col = e - b * m2;
                    const int64_t pos = 2 * (t0 + b);
                    if (col < m ? (pos == 0) : (pos + 1 >= a.Nl)) continue;
                    trsv_lower_col<MT, R, C>(sL + b * TRI, sInv + b * MT, sZ + b * MT * LDZ + col, LDZ, m);
                }
                __syncthreads();
            }
        }
    }

    // keep L (L^{-1} for kLinv), 1/diag(L) and Z for the solves
    bool bulk_l = false;
    if constexpr (kLinv) {
        // Z and (for even m) the rows of L^{-1} leave shared memory by bulk
        // asynchronous copies, which run under the Schur product below (it
        // reads sZ and writes neither region); waited for at the end
        bulk_l = (m & 1) == 0;
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            for (int b = 0; b < nbh; ++b) {
                const int64_t t = t0 + b, oz = t * 2 * (int64_t)mm, ol = t * (int64_t)mm;
                if (m == MT) {
                    if (CRS_IN(a, kDbgZ, oz) && CRS_IN(a, kDbgZ, oz + 2 * mm - 1))
                        bulk_s2g(a.Z + oz, sZ + b * MT * LDZ, (uint32_t)(2 * mm * sizeof(C)));
                } else {
                    for (int r = 0; r < m; ++r)
                        if (CRS_IN(a, kDbgZ, oz + r * m2) && CRS_IN(a, kDbgZ, oz + r * m2 + m2 - 1))
                            bulk_s2g(a.Z + oz + r * m2, sZ + (b * MT + r) * LDZ, (uint32_t)(m2 * sizeof(C)));
                }
                if (bulk_l)
                    for (int r = 0; r < m; ++r)
                        if (CRS_IN(a, kDbgL, ol + r * m) && CRS_IN(a, kDbgL, ol + r * m + m - 1))
                            bulk_s2g(a.L + ol + r * m, sLi + (b * MT + r) * kF32LdE, (uint32_t)(m * sizeof(C)));
            }
            asm volatile("cp.async.bulk.commit_group;" ::: "memory");
        }
    }
    if (!bulk_l) {
        for (int e = tid; e < nbh * mm; e += NT) {
            const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
            if (CRS_IN(a, kDbgL, (t0 + b) * mm + rem)) {
                C v = zmk(R(0), R(0));
                if (r >= c) {
                    if constexpr (kLinv) v = sLi[(b * MT + r) * kF32LdE + c];
                    else v = sL[b * TRI + tri(r, c)];
                }
                a.L[(t0 + b) * mm + rem] = v;
            }
        }
    }
    for (int e = tid; e < nbh * m; e += NT) {
        const int b = e / m, r = e - b * m;
        if (CRS_IN(a, kDbgInv, (t0 + b) * m + r)) a.inv[(t0 + b) * m + r] = sInv[b * MT + r];
    }
    if constexpr (!kLinv) {
        for (int e = tid; e < nbh * m * m2; e += NT) {
            const int b = e / (m * m2), rem = e - b * (m * m2), r = rem / m2, c = rem - r * m2;
            if (CRS_IN(a, kDbgZ, (t0 + b) * (int64_t)(m * m2) + rem))
                a.Z[(t0 + b) * (int64_t)(m * m2) + rem] = sZ[(b * MT + r) * LDZ + c];
        }
    }
    __syncthreads();

    // Lower triangle of Z^H Z.  Parts: Q^H Q is subtracted from the right
    // even block V_t in place, P^H P is kept in sW (the L buffer, free now) for
    // the left even block, and Q^H P = -F goes to the next level's B.
    C *sW = sL;
    if constexpr (std::is_same<R, float>::value && MT == 64) {
        // FP32 levels of the mixed form: on the tensor cores (tcgen05, TF32 x 3)
        unsigned char *stage = reinterpret_cast<unsigned char *>(
            (reinterpret_cast<uintptr_t>(sInv + (size_t)nb * MT) + 1023) & ~(uintptr_t)1023);
        if (tid == 0) {
            mbar_init(smem_u32(stage), 1);
            mbar_init(smem_u32(stage + 8), 1);
        }
        // three accumulators of 2MT = 128 columns
        if (tid < 32) tmem_alloc(smem_u32(stage + 16), 512);
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        uint32_t uses0 = 0, uses1 = 0, stage_count = 0;
        bool ok = true;
        for (int b = 0; b < nbh && ok; ++b)   // ok is the same in every thread
            ok = herk_tc_f32<MT>(a, t0 + b, sZ + b * MT * LDZ, sW + b * TRI, sV + b * TRI, stage, uses0, uses1,
                                 stage_count);
        if (tid < 32) tmem_dealloc(*reinterpret_cast<uint32_t *>(stage + 16), 512);
        if (!ok && tid == 0 && a.err) atomicExch(a.err, 1);
        __syncthreads();
    } else {
    // One item per entry.  The 2m real diagonal entries of each block come
    // first, in warps of their own (2 FMA per term instead of 4).
    const int ndiag = nbh * m2, dpadh = (ndiag + 31) & ~31, noff = m2 * (m2 - 1) / 2;
    for (int e = tid; e < dpadh + nbh * noff; e += NT) {
        if (e < ndiag) {
            const int b = e / m2, p = e - b * m2;
            const int64_t t = t0 + b;
            if (p < m ? (t == 0) : (2 * t + 1 >= a.Nl)) continue;
            const C *Zb = sZ + b * MT * LDZ + p;
            // the Q^H Q diagonal is accumulated straight into V (products
            // negated by a sign-bit XOR), the P^H P one from zero
            const bool intoV = p >= m;
            R *dst = intoV ? &sV[b * TRI + tri(p - m, p - m)].x : nullptr;
            R d = intoV ? *dst : R(0);
            const unsigned sg = intoV ? 0x80000000u : 0u;
#pragma unroll
            for (int s = 0; s < MT; ++s)
                if (s < m) {
                    const C v = Zb[s * LDZ];
                    d = fmx(flip_if(v.x, sg), v.x, d);
                    d = fmx(flip_if(v.y, sg), v.y, d);
                }
            if (intoV) *dst = d;
            else sW[b * TRI + tri(p, p)] = zmk(d, R(0));
        } else if (e >= dpadh) {
            const int e2 = e - dpadh, b = e2 / noff, g = e2 - b * noff;
            const int p = tri_row(g) + 1, q = g - p * (p - 1) / 2;   // p > q
            const int64_t t = t0 + b;
            const bool hasL = t >= 1, hasR = 2 * t + 1 < a.Nl;
            const int kind = (p < m) ? 0 : (q >= m ? 1 : 2);  // P^H P, Q^H Q, Q^H P
            if (kind == 0 ? !hasL : (kind == 1 ? !hasR : !(hasL && hasR))) continue;
            const C *Zb = sZ + b * MT * LDZ;
            // Q^H Q is accumulated straight into V and Q^H P into -F, their
            // products negated by a sign-bit XOR (no FP64 instruction, no
            // divergence between the kinds); P^H P from zero
            C *dst = kind == 1 ? &sV[b * TRI + tri(p - m, q - m)] : nullptr;
            C acc = dst ? *dst : zmk(R(0), R(0));
            const unsigned sg = kind == 0 ? 0u : 0x80000000u;
#pragma unroll
            for (int s = 0; s < MT; ++s)
                if (s < m) {
                    const C zp = Zb[s * LDZ + p];
                    zmac_ca(acc, zmk(flip_if(zp.x, sg), flip_if(zp.y, sg)), Zb[s * LDZ + q]);
                }
            if (kind == 0) {
                sW[b * TRI + tri(p, q)] = acc;
            } else if (kind == 1) {
                *dst = acc;
            } else if (CRS_IN(a, kDbgBn, (t - 1) * mm + (p - m) * m + q)) {
                a.Bn[(t - 1) * mm + (p - m) * m + q] = acc;
            }
        }
    }
    __syncthreads();
    }

    // V_j = (A_2j+1 - Q^H Q) - P^H P for the even blocks j = t0 + b.  The
    // CTA's last one misses its right neighbour's P^H P when that neighbour
    // starts the next CTA (k_factor_fix completes it); the CTA's first P^H P
    // goes to the boundary buffer for the previous CTA.
    const int nl = m * (m + 1) / 2;
    for (int e = tid; e < nbh * nl; e += NT) {
        const int b = e / nl, f = e - b * nl, r = tri_row(f), c = f - r * (r + 1) / 2;
        const int64_t j = t0 + b;
        if (b == 0 && j >= 1) {
            if (a.inline_fix) {
                // the previous chunk (same CTA, earlier) left V_{j-1} = A - Q^H Q
                const int64_t o = (j - 1) * mm;
                if (CRS_IN(a, kDbgAn, o + r * m + c) && CRS_IN(a, kDbgAn, o + c * m + r)) {
                    C v = zsub(a.An[o + r * m + c], sW[f]);
                    if (r == c) v.y = R(0);
                    a.An[o + r * m + c] = v;
                    if (r != c) a.An[o + c * m + r] = zconj(v);
                }
            } else if (CRS_IN(a, kDbgWbd, chunk * mm + r * m + c)) {
                a.Wbd[chunk * mm + r * m + c] = sW[f];
            }
        }
        if (j >= a.ne) continue;
        C v = sV[b * TRI + f];
        if (b + 1 < nbh) v = zsub(v, sW[(b + 1) * TRI + f]);
        if (CRS_IN(a, kDbgAn, j * mm + r * m + c)) a.An[j * mm + r * m + c] = v;
        if (r != c && CRS_IN(a, kDbgAn, j * mm + c * m + r)) a.An[j * mm + c * m + r] = zconj(v);
    }
    if (a.bd_count) {
        const int sec = bd_arrive(a.bd_count, chunk, crs_num_ctas(a.no, a.nb));
        for (int e = tid; e < ((sec & 1) ? nl : 0); e += NT) factor_fix_entry<R, true>(a, chunk, e);
        for (int e = tid; e < ((sec & 2) ? nl : 0); e += NT) factor_fix_entry<R, true>(a, chunk + 1, e);
    }
    // the bulk stores of L^{-1} and Z have read shared memory and written
    // global memory before the CTA ends (the hardware wait of the issuing thread)
    if constexpr (kLinv) {
        if (tid == 0) asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
    }
}

// Even block j = c * nb - 1 on the boundary between chunk c-1 and chunk c of
// a factor level: subtract P^H P of odd block c * nb, left by chunk c in
// Wbd[c].  Items e = first, first + stride, ... of (boundaries) * m(m+1)/2;
// the boundaries are c = 1 .. chunks-1, or with c_count > 0 the range
// c_begin .. c_begin + c_count - 1 (chunks c-1 and c must both be done).
template <class R>
__device__ __forceinline__ void factor_fix_items(const LevelArgsT<R> &a, int64_t first, int64_t stride) {
    const int nl = a.m * (a.m + 1) / 2;
    // boundaries c_first .. c_first + nbd - 1 (c_count = 0: all, 1 .. ncta - 1)
    const int64_t ncta = crs_num_ctas(a.no, a.nb);
    const int64_t c_first = a.c_count > 0 ? a.c_begin : 1, nbd = a.c_count > 0 ? a.c_count : ncta - 1;
    const int64_t total = nbd * nl;
    for (int64_t e = first; e < total; e += stride) {
        const int64_t c = c_first + e / nl;
        factor_fix_entry<R>(a, c, (int)(e - (c - c_first) * nl));
    }
}

// ------------------------------------------------------------- solve: down

// Entry rem (= row * k + column) of the boundary right-hand side of
// boundary c; kL2 as in factor_fix_entry.
template <class R, bool kL2 = false>
__device__ __forceinline__ void solve_down_fix_entry(const LevelArgsT<R> &a, int64_t c, int64_t rem) {
    const int64_t mk = (int64_t)a.m * a.k, j = c * a.nb - 1;
    if (!CRS_IN(a, kDbgYn, j * mk + rem) || !CRS_IN(a, kDbgCbd, c * mk + rem)) return;
    const auto *py = a.yn + j * mk + rem, *pc = a.cbd + c * mk + rem;
    a.yn[j * mk + rem] = kL2 ? zsub(__ldcg(py), __ldcg(pc)) : zsub(*py, *pc);
}

// One chunk of nb odd blocks and right-hand-side columns [cchunk*kc, +kc)
// of a down-sweep level, run by the whole CTA.
template <int MT, class R, bool kWide = false>
__device__ __forceinline__ void solve_down_chunk(const LevelArgsT<R> &a, int64_t chunk, int cchunk,
                                                 unsigned char *smem_raw) {
    using C = cplx_t<R>;
    constexpr int TRI = Tri<MT>::n;
    const int m = a.m, k = a.k, nb = a.nb, kc = a.kc, NT = blockDim.x, tid = threadIdx.x;
    const int mm = m * m, m2 = 2 * m, mk = m * k;
    const int c0 = cchunk * kc, kw = min(kc, k - c0);
    const int64_t t0 = chunk * nb;
    const int nbh = (int)min((int64_t)nb, a.no - t0);
    C *sL = reinterpret_cast<C *>(smem_raw);                           // [nb][TRI]
    C *sR = sL + (size_t)nb * TRI;                                       // [nb][MT][kc] r of odd t0+b
    C *sV = sR + (size_t)nb * MT * kc;                                   // [nb][MT][kc] v of even t0+b
    C *sW = sV + (size_t)nb * MT * kc;                                   // [nb][MT][kc] P^H r of odd t0+b
    R *sInv = reinterpret_cast<R *>(sW + (size_t)nb * MT * kc);  // [nb][MT]
    // FP32 with MT >= 32: Z is staged in shared memory too ([nb][MT][2MT]);
    // at FP32 speed its loads from L2 would otherwise dominate the products
    constexpr bool kStageZ = (sizeof(R) == 4 && MT >= 32);
    C *sZs = reinterpret_cast<C *>(sInv + (size_t)nb * MT + (((size_t)nb * MT) & 1));

    for (int e = tid; e < nbh * mm; e += NT) {
        const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
        if (r >= c) sL[b * TRI + tri(r, c)] = CRS_IN(a, kDbgL, (t0 + b) * mm + rem) ? a.L[(t0 + b) * mm + rem] : zmk(R(0), R(0));
    }
    for (int e = tid; e < nbh * m; e += NT) {
        const int b = e / m, r = e - b * m;
        sInv[b * MT + r] = CRS_IN(a, kDbgInv, (t0 + b) * m + r) ? a.inv[(t0 + b) * m + r] : R(0);
    }
    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        const int64_t t = t0 + b;
        const int64_t yo = (2 * t) * mk + r * k + c0 + c;
        sR[(b * MT + r) * kc + c] = CRS_IN(a, kDbgY, yo) ? a.y[yo] : zmk(R(0), R(0));
        if (t < a.ne) sV[(b * MT + r) * kc + c] = CRS_IN(a, kDbgY, yo + mk) ? a.y[yo + mk] : zmk(R(0), R(0));
    }
    if constexpr (kStageZ) {
        for (int e = tid; e < nbh * m * m2; e += NT) {
            const int b = e / (m * m2), rem = e - b * (m * m2), r = rem / m2, c = rem - r * m2;
            sZs[(b * MT + r) * 2 * MT + c] =
                CRS_IN(a, kDbgZ, (t0 + b) * (int64_t)(m * m2) + rem) ? a.Z[(t0 + b) * (int64_t)(m * m2) + rem] : zmk(R(0), R(0));
        }
    }
    __syncthreads();

    if constexpr (MT >= 32) {
        trsm_lower_cta<MT, R, C>(sL, sInv, sR, MT * kc, kc, nbh, kw, m);
    } else {
        if constexpr (kWide) {
            trsv_lower_wide<MT, R, C>(sL, sInv, sR, MT * kc, kc, nbh, kw, m, [](int, int) { return false; });
        } else {
            for (int e = tid; e < nbh * kw; e += NT) {
                const int b = e / kw, c = e - b * kw;
                trsv_lower_col<MT, R, C>(sL + b * TRI, sInv + b * MT, sR + b * MT * kc + c, kc, m);
            }
            __syncthreads();
        }
    }

    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        if (CRS_IN(a, kDbgR, (t0 + b) * mk + r * k + c0 + c)) a.r[(t0 + b) * mk + r * k + c0 + c] = sR[(b * MT + r) * kc + c];
    }
    // Z^H r: rows p < m give P^H r (kept in sW for the left even block), rows
    // p >= m give Q^H r (subtracted from the right even block in place)
    if constexpr (kStageZ) {
        // FP32: register tiles of 4 rows p x 2 columns c per thread (6 shared
        // loads per 8 complex FMAs instead of 2 per 1)
        constexpr int TP = 4, TC = 2;
        const int np = (m2 + TP - 1) / TP, ncl = (kw + TC - 1) / TC;
        for (int e = tid; e < nbh * np * ncl; e += NT) {
            const int b = e / (np * ncl), rem = e - b * (np * ncl), pt = rem / ncl, ct = rem - pt * ncl;
            const int p0 = pt * TP, cl0 = ct * TC;
            const C *Zs = sZs + b * MT * 2 * MT;
            const C *Rb = sR + b * MT * kc;
            C acc[TP][TC];
#pragma unroll
            for (int i = 0; i < TP; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) acc[i][j] = zmk(R(0), R(0));
            for (int s = 0; s < m; ++s) {
                C zv[TP], rv[TC];
#pragma unroll
                for (int i = 0; i < TP; ++i) zv[i] = (p0 + i < m2) ? Zs[s * 2 * MT + p0 + i] : zmk(R(0), R(0));
#pragma unroll
                for (int j = 0; j < TC; ++j) rv[j] = (cl0 + j < kw) ? Rb[s * kc + cl0 + j] : zmk(R(0), R(0));
#pragma unroll
                for (int i = 0; i < TP; ++i)
#pragma unroll
                    for (int j = 0; j < TC; ++j) zmac_ca(acc[i][j], zv[i], rv[j]);
            }
            const int64_t t = t0 + b;
#pragma unroll
            for (int i = 0; i < TP; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) {
                    const int p = p0 + i, c = cl0 + j;
                    if (p >= m2 || c >= kw) continue;
                    if (p < m) {
                        if (t >= 1) sW[(b * MT + p) * kc + c] = acc[i][j];
                    } else if (2 * t + 1 < a.Nl) {
                        C &v = sV[(b * MT + p - m) * kc + c];
                        v = zsub(v, acc[i][j]);
                    }
                }
        }
    } else {
        for (int e = tid; e < nbh * kw * m2; e += NT) {
            const int b = e / (kw * m2), rem = e - b * (kw * m2), c = rem / m2, p = rem - c * m2;
            const int64_t t = t0 + b;
            if (p < m ? (t == 0) : (2 * t + 1 >= a.Nl)) continue;
            const C *Rb = sR + b * MT * kc + c;
            const C *Zt = a.Z + t * (int64_t)(m * m2) + p;
            // Q^H r is accumulated straight into v, its products negated by a
            // sign-bit XOR; P^H r from zero
            C *dst = (p < m) ? &sW[(b * MT + p) * kc + c] : &sV[(b * MT + p - m) * kc + c];
            C acc = (p < m) ? zmk(R(0), R(0)) : *dst;
            const unsigned sg = (p < m) ? 0u : 0x80000000u;
#pragma unroll
            for (int s = 0; s < MT; ++s)
                if (s < m) {
                    const int64_t zo = t * (int64_t)(m * m2) + p + s * m2;
                    const C z = CRS_IN(a, kDbgZ, zo) ? __ldg(Zt + s * m2) : zmk(R(0), R(0));
                    zmac_ca(acc, zmk(flip_if(z.x, sg), flip_if(z.y, sg)), Rb[s * kc]);
                }
            *dst = acc;
        }
    }
    __syncthreads();
    // v_j = (y_2j+1 - Q^H r) - P^H r; the CTA's first P^H r goes to the boundary buffer
    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        const int64_t j = t0 + b;
        if (b == 0 && j >= 1) {
            if (a.inline_fix) {
                const int64_t o = (j - 1) * mk + r * k + c0 + c;
                if (CRS_IN(a, kDbgYn, o)) a.yn[o] = zsub(a.yn[o], sW[r * kc + c]);
            } else if (CRS_IN(a, kDbgCbd, chunk * mk + r * k + c0 + c)) {
                a.cbd[chunk * mk + r * k + c0 + c] = sW[r * kc + c];
            }
        }
        if (j >= a.ne) continue;
        C v = sV[(b * MT + r) * kc + c];
        if (b + 1 < nbh) v = zsub(v, sW[((b + 1) * MT + r) * kc + c]);
        if (CRS_IN(a, kDbgYn, j * mk + r * k + c0 + c)) a.yn[j * mk + r * k + c0 + c] = v;
    }
    if (a.bd_count) {
        // counters of this right-hand-side chunk: [cchunk][boundary]
        const int64_t ncta = crs_num_ctas(a.no, a.nb);
        const int sec = bd_arrive(a.bd_count + cchunk * ncta, chunk, ncta);
        for (int e = tid; e < ((sec & 1) ? m * kw : 0); e += NT)
            solve_down_fix_entry<R, true>(a, chunk, (e / kw) * k + c0 + e % kw);
        for (int e = tid; e < ((sec & 2) ? m * kw : 0); e += NT)
            solve_down_fix_entry<R, true>(a, chunk + 1, (e / kw) * k + c0 + e % kw);
    }
}

// Even block j = c * nb - 1 on a chunk boundary: subtract P^H r of odd block c * nb.
template <class R>
__device__ __forceinline__ void solve_down_fix_items(const LevelArgsT<R> &a, int64_t first, int64_t stride) {
    const int64_t mk = (int64_t)a.m * a.k, ncta = crs_num_ctas(a.no, a.nb), total = (ncta - 1) * mk;
    for (int64_t e = first; e < total; e += stride) {
        const int64_t c = 1 + e / mk;
        solve_down_fix_entry<R>(a, c, e - (c - 1) * mk);
    }
}

// --------------------------------------------------------------- solve: up

// One chunk of nb odd blocks and right-hand-side columns [cchunk*kc, +kc)
// of an up-sweep level, run by the whole CTA.
template <int MT, class R, bool kWide = false>
__device__ __forceinline__ void solve_up_chunk(const LevelArgsT<R> &a, int64_t chunk, int cchunk,
                                               unsigned char *smem_raw) {
    using C = cplx_t<R>;
    constexpr int TRI = Tri<MT>::n;
    const int m = a.m, k = a.k, nb = a.nb, kc = a.kc, NT = blockDim.x, tid = threadIdx.x;
    const int mm = m * m, m2 = 2 * m, mk = m * k;
    const int c0 = cchunk * kc, kw = min(kc, k - c0);
    const int64_t t0 = chunk * nb;
    const int nbh = (int)min((int64_t)nb, a.no - t0);
    C *sL = reinterpret_cast<C *>(smem_raw);                                // [nb][TRI]
    C *sW = sL + (size_t)nb * TRI;                                            // [nb][MT][kc]
    C *sX = sW + (size_t)nb * MT * kc;                                        // [nb][2MT][kc]
    R *sInv = reinterpret_cast<R *>(sX + (size_t)nb * 2 * MT * kc);  // [nb][MT]
    constexpr bool kStageZ = (sizeof(R) == 4 && MT >= 32);                     // see solve_down_chunk
    C *sZs = reinterpret_cast<C *>(sInv + (size_t)nb * MT + (((size_t)nb * MT) & 1));

    if (a.level == 0 && *a.status != CRS_NO_FAIL) {
        // the factorisation broke down: the result is NaN
        const C nan2 = zmk(qnan(R()), qnan(R()));
        for (int e = tid; e < nbh * m * kw; e += NT) {
            const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
            const int64_t t = t0 + b;
            if (CRS_IN(a, kDbgX, (2 * t) * mk + r * k + c0 + c)) a.x[(2 * t) * mk + r * k + c0 + c] = nan2;
            if (t < a.ne && CRS_IN(a, kDbgX, (2 * t + 1) * mk + r * k + c0 + c))
                a.x[(2 * t + 1) * mk + r * k + c0 + c] = nan2;
        }
        return;
    }

    for (int e = tid; e < nbh * mm; e += NT) {
        const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
        if (r >= c) sL[b * TRI + tri(r, c)] = CRS_IN(a, kDbgL, (t0 + b) * mm + rem) ? a.L[(t0 + b) * mm + rem] : zmk(R(0), R(0));
    }
    for (int e = tid; e < nbh * m; e += NT) {
        const int b = e / m, r = e - b * m;
        sInv[b * MT + r] = CRS_IN(a, kDbgInv, (t0 + b) * m + r) ? a.inv[(t0 + b) * m + r] : R(0);
    }
    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        const int64_t t = t0 + b;
        const int64_t ro = t * mk + r * k + c0 + c;
        sW[(b * MT + r) * kc + c] = CRS_IN(a, kDbgR, ro) ? a.r[ro] : zmk(R(0), R(0));
        // [x_left; x_right] = [xn_{t-1}; xn_t], zero past the boundary
        sX[(b * 2 * MT + r) * kc + c] = (t >= 1 && CRS_IN(a, kDbgXn, ro - mk)) ? a.xn[ro - mk] : zmk(R(0), R(0));
        const C xr = (t < a.ne && CRS_IN(a, kDbgXn, ro)) ? a.xn[ro] : zmk(R(0), R(0));
        sX[(b * 2 * MT + m + r) * kc + c] = xr;
        if (t < a.ne && CRS_IN(a, kDbgX, (2 * t + 1) * mk + r * k + c0 + c))
            a.x[(2 * t + 1) * mk + r * k + c0 + c] = xr;  // even unknowns
    }
    if constexpr (kStageZ) {
        for (int e = tid; e < nbh * m * m2; e += NT) {
            const int b = e / (m * m2), rem = e - b * (m * m2), r = rem / m2, c = rem - r * m2;
            sZs[(b * MT + r) * 2 * MT + c] =
                CRS_IN(a, kDbgZ, (t0 + b) * (int64_t)(m * m2) + rem) ? a.Z[(t0 + b) * (int64_t)(m * m2) + rem] : zmk(R(0), R(0));
        }
    }
    __syncthreads();

    // w = r - P x_left - Q x_right
    if constexpr (kStageZ) {
        // FP32: register tiles of 2 rows x 2 columns per thread
        constexpr int TR = 2, TC = 2;
        const int nrt = (m + TR - 1) / TR, ncl = (kw + TC - 1) / TC;
        for (int e = tid; e < nbh * nrt * ncl; e += NT) {
            const int b = e / (nrt * ncl), rem = e - b * (nrt * ncl), rt = rem / ncl, ct = rem - rt * ncl;
            const int r0 = rt * TR, cl0 = ct * TC;
            const C *Zs = sZs + b * MT * 2 * MT;
            const C *Xb = sX + b * 2 * MT * kc;
            C acc[TR][TC];
#pragma unroll
            for (int i = 0; i < TR; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j)
                    acc[i][j] = (r0 + i < m && cl0 + j < kw) ? sW[(b * MT + r0 + i) * kc + cl0 + j] : zmk(R(0), R(0));
            for (int s = 0; s < m2; ++s) {
                C zv[TR], xv[TC];
#pragma unroll
                for (int i = 0; i < TR; ++i) zv[i] = (r0 + i < m) ? Zs[(r0 + i) * 2 * MT + s] : zmk(R(0), R(0));
#pragma unroll
                for (int j = 0; j < TC; ++j) xv[j] = (cl0 + j < kw) ? Xb[s * kc + cl0 + j] : zmk(R(0), R(0));
#pragma unroll
                for (int i = 0; i < TR; ++i)
#pragma unroll
                    for (int j = 0; j < TC; ++j) zmsub(acc[i][j], zv[i], xv[j]);
            }
#pragma unroll
            for (int i = 0; i < TR; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j)
                    if (r0 + i < m && cl0 + j < kw) sW[(b * MT + r0 + i) * kc + cl0 + j] = acc[i][j];
        }
    } else {
        for (int e = tid; e < nbh * m * kw; e += NT) {
            const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
            const int64_t t = t0 + b;
            const C *Xb = sX + b * 2 * MT * kc + c;
            C acc = sW[(b * MT + r) * kc + c];
            const C *Zr = a.Z + t * (int64_t)(m * m2) + r * m2;
#pragma unroll
            for (int s = 0; s < 2 * MT; ++s)
                if (s < m2 && CRS_IN(a, kDbgZ, t * (int64_t)(m * m2) + r * m2 + s)) zmsub(acc, __ldg(Zr + s), Xb[s * kc]);
            sW[(b * MT + r) * kc + c] = acc;
        }
    }
    __syncthreads();

    // x_odd = L^{-H} w
    if constexpr (MT >= 32) {
        trsm_lower_h_cta<MT, R, C>(sL, sInv, sW, MT * kc, kc, nbh, kw, m);
    } else {
        if constexpr (kWide) {
            trsv_lower_h_wide<MT, R, C>(sL, sInv, sW, MT * kc, kc, nbh, kw, m);
        } else {
            for (int e = tid; e < nbh * kw; e += NT) {
                const int b = e / kw, c = e - b * kw;
                trsv_lower_h_col<MT, R, C>(sL + b * TRI, sInv + b * MT, sW + b * MT * kc + c, kc, m);
            }
            __syncthreads();
        }
    }
    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        if (CRS_IN(a, kDbgX, (2 * (t0 + b)) * mk + r * k + c0 + c))
            a.x[(2 * (t0 + b)) * mk + r * k + c0 + c] = sW[(b * MT + r) * kc + c];
    }
}

}  // namespace crs
