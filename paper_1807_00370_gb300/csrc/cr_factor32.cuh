// cr_factor32.cuh -- Cholesky factor, its inverse and Z of one odd block for
// the FP32 levels of the mixed-precision form, block size class MT = 64, by
// 16 x 16 blocks (included by cr_core.cuh).
//
// For one odd block of a level (Sec. 2, eq. Formulas) the factorisation needs
// A = L L^H (with the breakdown test on every pivot), Z = L^{-1} [B_l | B_r^H]
// and, for the product form of the FP32 sweeps (cr_solve32.cu), E = L^{-1}.
// Here all three are built from 16 x 16 blocks, so that the dependent chains
// are at most 16 steps long and sit inside one warp, and the rest is
// products with independent outputs:
//   for each panel p (columns 16p .. 16p + 15):
//     1. one warp factors the diagonal block D = L_pp in registers (row
//        16p + lane in lane; right-looking: pivot from lane c, column c
//        scaled, rank-1 update of the rows below with the entries L[j][c]
//        from lane j by shuffles) and, in the same steps, forms
//        E_pp = D^{-1} row by row (forward substitution on the identity);
//     2. the rows below take L_ip = A_ip E_pp^H;
//     3. the trailing lower triangle is updated, A_ij -= L_ip L_jp^H;
//   then the blocks of E below the diagonal, by distance d = i - j:
//     E_ij = -E_ii sum_{k=j}^{i-1} L_ik E_kj;
//   and finally Z = E [B_l | B_r^H] as one product (E lower triangular).
// The pivots and the breakdown test are those of the column-by-column
// factorisation: d = A_cc - sum |L_cs|^2 must be > 0 (a NaN fails).
#pragma once

namespace crs {

constexpr int kF32LdE = 64 + 2;   // row of E in shared memory (complex), 16-byte padded

__device__ __forceinline__ void f32_cp8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}
// Bulk asynchronous copy of `bytes` (a multiple of 16; both addresses
// 16-byte aligned) from shared to global memory, in the issuing thread's
// bulk group.
__device__ __forceinline__ void bulk_s2g(void *gdst, const void *ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"((uint32_t)__cvta_generic_to_shared(ssrc)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void f32_cp16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
                 : "memory");
}

// Staging of a chunk's blocks for the FP32 factor of class MT = 64: the
// lower triangles of A_2t (-> sL) and A_2t+1 (-> sV, real diagonal) and
// B_{2t-1} (-> the P columns of sZ) are plain copies and go by cp.async
// (none of them passes through registers); B_{2t}^H (-> the Q columns of sZ)
// is a transpose, loaded into registers with consecutive threads on
// consecutive rows of B_{2t}, so that the transposed stores fall on
// consecutive words.  Blocks without a left (right) neighbour get zero P (Q).
// Ends with __syncthreads().
template <int MT>
__device__ __forceinline__ void stage_f32_64(const LevelArgsT<float> &a, int64_t t0, int nbh, float2 *sL, float2 *sV,
                                             float2 *sZ) {
    constexpr int TRI = MT * (MT + 1) / 2, LDZ = 2 * MT;
    const int m = a.m, NT = blockDim.x, tid = threadIdx.x, nl = m * (m + 1) / 2;
    const int64_t mm = (int64_t)m * m;
    const float2 zero = make_float2(0.f, 0.f);
    for (int b = 0; b < nbh; ++b) {
        const int64_t t = t0 + b, pos = 2 * t;
        for (int f = tid; f < nl; f += NT) {
            const int r = tri_row(f), c = f - r * (r + 1) / 2;
            const int64_t o = pos * mm + r * m + c;
            if (CRS_IN(a, kDbgA, o)) f32_cp8(sL + b * TRI + f, a.A + o);
            if (t < a.ne && CRS_IN(a, kDbgA, o + mm)) f32_cp8(sV + b * TRI + f, a.A + o + mm);
        }
        float2 *Zb = sZ + b * MT * LDZ;
        if (pos >= 1) {
            const int64_t o = (pos - 1) * mm;
            if ((m & 1) == 0) {
                const int h = m / 2;
                for (int e = tid; e < m * h; e += NT) {
                    const int r = e / h, g = e - r * h;
                    if (CRS_IN(a, kDbgB, o + r * m + 2 * g) && CRS_IN(a, kDbgB, o + r * m + 2 * g + 1))
                        f32_cp16(Zb + r * LDZ + 2 * g, a.B + o + r * m + 2 * g);
                }
            } else {
                for (int e = tid; e < m * m; e += NT) {
                    const int r = e / m, c = e - r * m;
                    if (CRS_IN(a, kDbgB, o + e)) f32_cp8(Zb + r * LDZ + c, a.B + o + e);
                }
            }
        } else {
            for (int e = tid; e < m * m; e += NT) Zb[(e / m) * LDZ + e % m] = zero;
        }
        if (pos + 1 < a.Nl) {
            const int64_t o = pos * mm;
            const int ncq = (m + 3) / 4;
            for (int e = tid; e < m * ncq; e += NT) {
                const int r = e % m, cq = e / m;   // consecutive threads: consecutive rows r
                float2 v[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = 4 * cq + i;
                    v[i] = (c < m && CRS_IN(a, kDbgB, o + r * m + c)) ? __ldg(a.B + o + r * m + c) : zero;
                }
#pragma unroll
                for (int i = 0; i < 4; ++i) {
                    const int c = 4 * cq + i;
                    if (c < m) Zb[c * LDZ + m + r] = zconj(v[i]);
                }
            }
        } else {
            for (int e = tid; e < m * m; e += NT) Zb[(e % m) * LDZ + m + e / m] = zero;
        }
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int e = tid; e < nbh * m; e += NT) {   // the diagonal of A_2t+1 is real
        const int b = e / m, r = e - b * m;
        if (t0 + b < a.ne) sV[b * TRI + tri(r, r)].y = 0.f;
    }
    __syncthreads();
}

// One block, run by the whole CTA.  Lb: packed lower triangle of A (in: the
// odd diagonal block; out: L); ivb[MT]: 1 / diag(L); E: [MT][kF32LdE], all
// zero on entry (out: L^{-1}, zero above the diagonal); Zb: [MT][2MT] (in:
// [B_l | B_r^H]; out: Z).  `fail_index` is the 1-based block index a
// breakdown reports.  Ends with __syncthreads().
template <int MT>
__device__ __forceinline__ void chol_inv_z_f32(const LevelArgsT<float> &a, int64_t fail_index, float2 *Lb, float *ivb,
                                               float2 *E, float2 *Zb) {
    static_assert(MT == 64, "blocked FP32 factor: class MT = 64");
    using C = float2;
    constexpr int LDZ = 2 * MT, LDE = kF32LdE;
    const int m = a.m, m2 = 2 * m, NT = blockDim.x, tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int nbk = (m + 15) / 16;
    const C zero = make_float2(0.f, 0.f);

    for (int p = 0; p < nbk; ++p) {
        const int kb = 16 * p, w = min(16, m - kb);
        // 1. diagonal block (warp 0): D = L_pp and its inverse E_pp together.
        // Lane r holds row r of D and row r of E_pp.  At step c lane c's pivot
        // d = A_cc - sum |L_cs|^2 is final; its rows of D and E are scaled by
        // 1 / sqrt(d), lanes r > c scale L[r][c]; then column c of D and row c
        // of E (both from lane c's step) are shuffled to every lane, and lane
        // r > c updates L[r][j] -= L[r][c] conj(L[j][c]) (j in (c, r]) and
        // E[r][j] -= L[r][c] E[c][j] (j <= c): forward substitution on the
        // identity, row by row, alongside the factorisation.
        if (warp == 0) {
            C row[16], er[16];
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                row[j] = (lane < w && j <= lane) ? Lb[tri(kb + lane, kb + j)] : zero;
                er[j] = make_float2((lane < w && j == lane) ? 1.f : 0.f, 0.f);
            }
#pragma unroll
            for (int c = 0; c < 16; ++c) {
                if (c < w) {   // the same in every lane
                    const float d = __shfl_sync(0xffffffffu, row[c].x, c);
                    if (lane == c && !(d > 0.f)) report_fail(a.status, a.level, fail_index);
                    const float iv = rsq(d);
                    if (lane == c) {
                        row[c] = make_float2(d * iv, 0.f);
                        ivb[kb + c] = iv;
#pragma unroll
                        for (int j = 0; j <= c; ++j) er[j] = zscale(er[j], iv);
                    } else if (lane > c) {
                        row[c] = zscale(row[c], iv);
                    }
                    // all shuffles of the step first, so that their latencies overlap
                    C lj[16], ec[16];
#pragma unroll
                    for (int j = c + 1; j < 16; ++j)
                        lj[j] = make_float2(__shfl_sync(0xffffffffu, row[c].x, j), __shfl_sync(0xffffffffu, row[c].y, j));
#pragma unroll
                    for (int j = 0; j <= c; ++j)
                        ec[j] = make_float2(__shfl_sync(0xffffffffu, er[j].x, c), __shfl_sync(0xffffffffu, er[j].y, c));
#pragma unroll
                    for (int j = c + 1; j < 16; ++j)
                        if (j < w && lane >= j) zmsub_cb(row[j], row[c], lj[j]);   // L[r][j] -= L[r][c] conj(L[j][c])
                    if (lane > c && lane < w) {
#pragma unroll
                        for (int j = 0; j <= c; ++j) zmsub(er[j], row[c], ec[j]);   // E[r][j] -= L[r][c] E[c][j]
                    }
                }
            }
            if (lane < w) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    if (j <= lane) {
                        Lb[tri(kb + lane, kb + j)] = row[j];
                        E[(kb + lane) * LDE + kb + j] = er[j];
                    }
                }
            }
        }
        __syncthreads();
        // 2. rows below: L[r][kb + c] = sum_{j <= c} A[r][kb + j] conj(E_pp[c][j]),
        // four threads per row (columns g, g + 4, g + 8, g + 12), results kept
        // in registers until every thread of the row has read it
        {
            const int nbel = m - kb - w;
            const int r = kb + w + (tid >> 2), g = tid & 3;
            const bool act = tid < 4 * nbel;
            C y[4];
            if (act) {
                C x[16];
#pragma unroll
                for (int j = 0; j < 16; ++j) x[j] = j < w ? Lb[tri(r, kb + j)] : zero;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = g + 4 * q;
                    const C *Ec = E + (kb + c) * LDE + kb;
                    C acc = zero;
#pragma unroll
                    for (int j = 0; j < 16; ++j)
                        if (j <= c) zmac_cb(acc, x[j], Ec[j]);
                    y[q] = acc;
                }
            }
            __syncthreads();
            if (act) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (g + 4 * q < w) Lb[tri(r, kb + g + 4 * q)] = y[q];
            }
        }
        __syncthreads();
        // 3. trailing update: A[r][q] -= sum_{j in panel} L[r][j] conj(L[q][j]), kb + w <= q <= r < m
        const int ke = kb + w;
        if (ke < m) {
            const int nr = m - ke, ntr = nr * (nr + 1) / 2;
            for (int f = tid; f < ntr; f += NT) {
                const int rr = tri_row(f), qq = f - rr * (rr + 1) / 2;
                const int r = ke + rr, q = ke + qq;
                const C *Lr = Lb + tri(r, kb), *Lq = Lb + tri(q, kb);
                C u = Lb[tri(r, q)];
#pragma unroll
                for (int j = 0; j < 16; ++j) zmsub_cb(u, Lr[j], Lq[j]);
                Lb[tri(r, q)] = u;
            }
            __syncthreads();
        }
    }

    // E below the diagonal, by block distance d: S = sum_{k=j}^{i-1} L_ik E_kj
    // into the (zero) block E_ij, then E_ij = -E_ii S in place (a thread per
    // column, rows from the bottom so that S[t][c], t <= r, is still there)
    for (int d = 1; d < nbk; ++d) {
        const int npair = nbk - d;
        for (int e = tid; e < npair * 256; e += NT) {
            const int j = e >> 8, i = j + d, r = (e >> 4) & 15, c = e & 15;
            const int gr = 16 * i + r, gc = 16 * j + c;
            if (gr >= m || gc >= m) continue;
            C acc = zero;
            for (int k = j; k < i; ++k) {
                const C *Lr = Lb + tri(gr, 16 * k);
                const int wk = min(16, m - 16 * k);
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (u < wk) zmac(acc, Lr[u], E[(16 * k + u) * LDE + gc]);
            }
            E[gr * LDE + gc] = acc;
        }
        __syncthreads();
        for (int e = tid; e < npair * 16; e += NT) {
            const int j = e >> 4, i = j + d, c = e & 15;
            const int gc = 16 * j + c, wi = min(16, m - 16 * i);
            if (gc >= m) continue;
            C s[16];
#pragma unroll
            for (int t = 0; t < 16; ++t) s[t] = t < wi ? E[(16 * i + t) * LDE + gc] : zero;
#pragma unroll
            for (int r = 15; r >= 0; --r) {
                if (r < wi) {
                    const C *Er = E + (16 * i + r) * LDE + 16 * i;
                    C acc = zero;
#pragma unroll
                    for (int t = 0; t <= r; ++t) zmac(acc, Er[t], s[t]);
                    E[(16 * i + r) * LDE + gc] = zneg(acc);
                }
            }
        }
        __syncthreads();
    }

    // Z = E [B_l | B_r^H]: thread tile of 4 rows x 8 columns (16 row groups x
    // 16 column groups), s <= last row of the tile (E lower triangular); the
    // products are kept in registers until every thread has read Zb.  Warp w
    // takes rows 8 rb .. 8 rb + 7 with rb = w for w < 4 and 11 - w otherwise,
    // so that warps w and w + 4 (one scheduler) share 9 of the 36 units of
    // the triangle.
    {
        const int wz = tid >> 5, rbz = wz < 4 ? wz : 11 - wz;
        const int cg = tid & 15, rg = 2 * rbz + ((tid >> 4) & 1);
        C acc[4][8];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int q = 0; q < 8; ++q) acc[i][q] = zero;
        if (NT >= 256 && rg < 16) {
            const int r0 = 4 * rg, c0 = 8 * cg, s1 = min(m, r0 + 4);
            for (int s = 0; s < s1; ++s) {
                C ev[4], bv[8];
#pragma unroll
                for (int i = 0; i < 4; ++i) ev[i] = E[(r0 + i) * LDE + s];
#pragma unroll
                for (int q = 0; q < 8; q += 2) {
                    const float4 v = *reinterpret_cast<const float4 *>(Zb + s * LDZ + c0 + q);
                    bv[q] = make_float2(v.x, v.y);
                    bv[q + 1] = make_float2(v.z, v.w);
                }
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int q = 0; q < 8; ++q) zmac(acc[i][q], ev[i], bv[q]);
            }
        }
        __syncthreads();
        if (NT >= 256 && rg < 16) {
            const int r0 = 4 * rg, c0 = 8 * cg;
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (r0 + i < m && c0 + q < m2) Zb[(r0 + i) * LDZ + c0 + q] = acc[i][q];
        }
        __syncthreads();
    }
}

}  // namespace crs
