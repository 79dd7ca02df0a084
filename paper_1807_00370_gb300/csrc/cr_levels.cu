// cr_levels.cu -- the per-level kernels of classic cyclic reduction in FP64.
//
// One level (Sec. 2, eq. Formulas; 0-based: odd block t at position 2t, even
// block j' at 2j'+1):
//   k_factor_odd   per odd block: Cholesky A_2t = L L^H with the breakdown
//                  test, Z = [P | Q] = L^{-1} [B_{2t-1} | B_{2t}^H], and the
//                  Hermitian product Z^H Z (Sec. 4's rule), whose three parts
//                  are P^H P (to the left even block), Q^H Q (to the right
//                  even block) and Q^H P (= -F, the next level's B).
//   k_factor_even  per even block: V = A_{2j'+1} - Q^H Q(left) - P^H P(right).
//   k_solve_down_* r = L^{-1} y_odd, then v = y_even - Q^H r(left) - P^H r(right).
//   k_solve_up     x_odd = L^{-H}(r - P x_left - Q x_right); x_even copied.
//
// GPU mapping.  A CTA owns nb consecutive odd blocks and stages them in
// shared memory.  Each phase is a list of equal-cost work items (a matrix
// entry, a column of a triangular solve) spread over all threads of the CTA,
// so that warps issue FP64 instructions with every lane active: on GB300 the
// FP64 pipe (2 DFMA/clk/SM) is the bound of this path, and one warp per SM
// sub-partition with a dependent chain already keeps it ~90% busy, so
// occupancy matters little and lane utilisation and instruction count matter
// most.
#include "cr_launch.h"

namespace crs {

// --------------------------------------------------------------- helpers

// z := L^{-1} z for one column z (shared memory, stride ld).
template <int MT>
__device__ __forceinline__ void trsv_lower_col(const z2 *Lb, const double *ivb, z2 *col, int ld, int m) {
    if constexpr (MT <= 32) {
        z2 z[MT];
#pragma unroll
        for (int r = 0; r < MT; ++r)
            if (r < m) z[r] = col[r * ld];
#pragma unroll
        for (int r = 0; r < MT; ++r) {
            if (r < m) {
                z2 acc = z[r];
#pragma unroll
                for (int s = 0; s < r; ++s) zmsub(acc, Lb[r * MT + s], z[s]);
                z[r] = zscale(acc, ivb[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < MT; ++r)
            if (r < m) col[r * ld] = z[r];
    } else {
        for (int r = 0; r < m; ++r) {
            z2 acc = col[r * ld];
            for (int s = 0; s < r; ++s) zmsub(acc, Lb[r * MT + s], col[s * ld]);
            col[r * ld] = zscale(acc, ivb[r]);
        }
    }
}

// z := L^{-H} z for one column z (shared memory, stride ld).
template <int MT>
__device__ __forceinline__ void trsv_lower_h_col(const z2 *Lb, const double *ivb, z2 *col, int ld, int m) {
    if constexpr (MT <= 32) {
        z2 z[MT];
#pragma unroll
        for (int r = 0; r < MT; ++r)
            if (r < m) z[r] = col[r * ld];
#pragma unroll
        for (int r = MT - 1; r >= 0; --r) {
            if (r < m) {
                z2 acc = z[r];
#pragma unroll
                for (int s = r + 1; s < MT; ++s)
                    if (s < m) zmsub_ca(acc, Lb[s * MT + r], z[s]);
                z[r] = zscale(acc, ivb[r]);
            }
        }
#pragma unroll
        for (int r = 0; r < MT; ++r)
            if (r < m) col[r * ld] = z[r];
    } else {
        for (int r = m - 1; r >= 0; --r) {
            z2 acc = col[r * ld];
            for (int s = r + 1; s < m; ++s) zmsub_ca(acc, Lb[s * MT + r], col[s * ld]);
            col[r * ld] = zscale(acc, ivb[r]);
        }
    }
}

// ------------------------------------------------------------ factor: odd

template <int MT>
__global__ void __launch_bounds__(256) k_factor_odd(LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int LDZ = 2 * MT;
    const int m = a.m, nb = a.nb, NT = blockDim.x, tid = threadIdx.x;
    const int mm = m * m, m2 = 2 * m;
    const int64_t t0 = (int64_t)blockIdx.x * nb;
    const int nbh = (int)min((int64_t)nb, a.no - t0);
    z2 *sL = reinterpret_cast<z2 *>(smem_raw);                          // [nb][MT][MT]
    z2 *sZ = sL + (size_t)nb * MT * MT;                                  // [nb][MT][2MT]
    double *sInv = reinterpret_cast<double *>(sZ + (size_t)nb * MT * LDZ);  // [nb][MT]

    // stage the lower triangle of A_2t, B_{2t-1} (P part) and B_{2t}^H (Q part)
    for (int e = tid; e < nbh * mm; e += NT) {
        const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
        const int64_t pos = 2 * (t0 + b);
        sL[(b * MT + r) * MT + c] = (r >= c) ? a.A[pos * mm + rem] : zmk(0.0, 0.0);
        sZ[(b * MT + r) * LDZ + c] = (pos >= 1) ? a.B[(pos - 1) * mm + rem] : zmk(0.0, 0.0);
        sZ[(b * MT + c) * LDZ + m + r] = (pos + 1 < a.Nl) ? zconj(a.B[pos * mm + rem]) : zmk(0.0, 0.0);
    }
    __syncthreads();

    // Cholesky, left-looking by columns.  Pass 1 of column c: the pivots
    // (one item per block, in warps of their own so that the sqrt path does
    // not diverge from the off-diagonal path), then the unscaled entries
    // below the pivot.  Pass 2 scales them by 1 / pivot.
    const int dpad = (nbh + 31) & ~31;
    for (int c = 0; c < m; ++c) {
        const int below = m - c - 1;
        for (int e = tid; e < dpad + nbh * below; e += NT) {
            if (e < nbh) {
                const int b = e;
                z2 *Lb = sL + b * MT * MT;
                double d = Lb[c * MT + c].x;
                for (int s = 0; s < c; ++s) {
                    const z2 l = Lb[c * MT + s];
                    d = fma(-l.x, l.x, d);
                    d = fma(-l.y, l.y, d);
                }
                if (!(d > 0.0)) report_fail(a.status, a.level, 2 * (t0 + b) + 1);
                const double iv = rsqrt(d);
                sInv[b * MT + c] = iv;
                Lb[c * MT + c] = zmk(d * iv, 0.0);
            } else if (e >= dpad) {
                const int e2 = e - dpad, b = e2 / below, r = c + 1 + (e2 - b * below);
                z2 *Lb = sL + b * MT * MT;
                z2 u = Lb[r * MT + c];
                for (int s = 0; s < c; ++s) zmsub_cb(u, Lb[r * MT + s], Lb[c * MT + s]);
                Lb[r * MT + c] = u;
            }
        }
        __syncthreads();
        for (int e = tid; e < nbh * below; e += NT) {
            const int b = e / below, r = c + 1 + (e - b * below);
            z2 *p = sL + (b * MT + r) * MT + c;
            *p = zscale(*p, sInv[b * MT + c]);
        }
        __syncthreads();
    }

    // Z := L^{-1} Z, one item per (block, column); zero columns stay zero
    for (int e = tid; e < nbh * m2; e += NT) {
        const int b = e / m2, col = e - b * m2;
        const int64_t pos = 2 * (t0 + b);
        if (col < m ? (pos == 0) : (pos + 1 >= a.Nl)) continue;
        trsv_lower_col<MT>(sL + b * MT * MT, sInv + b * MT, sZ + b * MT * LDZ + col, LDZ, m);
    }
    __syncthreads();

    // keep L, 1/diag(L) and Z for the solves
    for (int e = tid; e < nbh * mm; e += NT) {
        const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
        a.L[(t0 + b) * mm + rem] = (r >= c) ? sL[(b * MT + r) * MT + c] : zmk(0.0, 0.0);
    }
    for (int e = tid; e < nbh * m; e += NT) {
        const int b = e / m, r = e - b * m;
        a.inv[(t0 + b) * m + r] = sInv[b * MT + r];
    }
    for (int e = tid; e < nbh * m * m2; e += NT) {
        const int b = e / (m * m2), rem = e - b * (m * m2), r = rem / m2, c = rem - r * m2;
        a.Z[(t0 + b) * (int64_t)(m * m2) + rem] = sZ[(b * MT + r) * LDZ + c];
    }

    // Lower triangle of Z^H Z.  The 2m real diagonal entries of each block
    // come first, in warps of their own (2 FMA per term instead of 4), then
    // the strictly lower entries (one complex dot product of length m each).
    // Parts: rows/cols < m give P^H P, both >= m give Q^H Q, row >= m > col
    // gives Q^H P = -F.
    const int ndiag = nbh * m2, dpadh = (ndiag + 31) & ~31, noff = m2 * (m2 - 1) / 2;
    for (int e = tid; e < dpadh + nbh * noff; e += NT) {
        if (e < ndiag) {
            const int b = e / m2, p = e - b * m2;
            const int64_t t = t0 + b, pos = 2 * t;
            if (p < m ? (pos == 0) : (pos + 1 >= a.Nl)) continue;
            const z2 *Zb = sZ + b * MT * LDZ;
            double d = 0.0;
#pragma unroll
            for (int s = 0; s < MT; ++s)
                if (s < m) {
                    const z2 v = Zb[s * LDZ + p];
                    d = fma(v.x, v.x, d);
                    d = fma(v.y, v.y, d);
                }
            if (p < m) a.Wl[t * mm + p * m + p] = zmk(d, 0.0);
            else a.Wr[t * mm + (p - m) * m + (p - m)] = zmk(d, 0.0);
        } else if (e >= dpadh) {
            const int e2 = e - dpadh, b = e2 / noff, g = e2 - b * noff;
            const int p = tri_row(g) + 1, q = g - p * (p - 1) / 2;   // p > q
            const int64_t t = t0 + b, pos = 2 * t;
            const bool hasL = pos >= 1, hasR = pos + 1 < a.Nl;
            const int kind = (p < m) ? 0 : (q >= m ? 1 : 2);  // P^H P, Q^H Q, Q^H P
            if (kind == 0 ? !hasL : (kind == 1 ? !hasR : !(hasL && hasR))) continue;
            const z2 *Zb = sZ + b * MT * LDZ;
            z2 acc = zmk(0.0, 0.0);
#pragma unroll
            for (int s = 0; s < MT; ++s)
                if (s < m) zmac_ca(acc, Zb[s * LDZ + p], Zb[s * LDZ + q]);
            if (kind == 0) a.Wl[t * mm + p * m + q] = acc;
            else if (kind == 1) a.Wr[t * mm + (p - m) * m + (q - m)] = acc;
            else a.Bn[(t - 1) * mm + (p - m) * m + q] = zneg(acc);
        }
    }
}

// ----------------------------------------------------------- factor: even

__global__ void __launch_bounds__(256) k_factor_even(LevelArgs a) {
    const int m = a.m, mm = m * m, nl = m * (m + 1) / 2;
    const int64_t total = a.ne * nl;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / nl;
        const int f = (int)(e - j * nl);
        const int p = tri_row(f), q = f - p * (p + 1) / 2;
        z2 v = a.A[(2 * j + 1) * mm + p * m + q];
        v = zsub(v, a.Wr[j * mm + p * m + q]);                       // Q^H Q of odd block j (left)
        if (j + 1 < a.no) v = zsub(v, a.Wl[(j + 1) * mm + p * m + q]);  // P^H P of odd block j+1 (right)
        if (p == q) v.y = 0.0;
        a.An[j * mm + p * m + q] = v;
        if (p != q) a.An[j * mm + q * m + p] = zconj(v);
    }
}

// ------------------------------------------------------------- solve: down

template <int MT>
__global__ void __launch_bounds__(256) k_solve_down_odd(LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = a.m, k = a.k, nb = a.nb, kc = a.kc, NT = blockDim.x, tid = threadIdx.x;
    const int mm = m * m, m2 = 2 * m, mk = m * k;
    const int c0 = blockIdx.y * kc, kw = min(kc, k - c0);
    const int64_t t0 = (int64_t)blockIdx.x * nb;
    const int nbh = (int)min((int64_t)nb, a.no - t0);
    z2 *sL = reinterpret_cast<z2 *>(smem_raw);                           // [nb][MT][MT]
    z2 *sR = sL + (size_t)nb * MT * MT;                                   // [nb][MT][kc]
    double *sInv = reinterpret_cast<double *>(sR + (size_t)nb * MT * kc);  // [nb][MT]

    for (int e = tid; e < nbh * mm; e += NT) {
        const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
        sL[(b * MT + r) * MT + c] = a.L[(t0 + b) * mm + rem];
    }
    for (int e = tid; e < nbh * m; e += NT) {
        const int b = e / m, r = e - b * m;
        sInv[b * MT + r] = a.inv[(t0 + b) * m + r];
    }
    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        sR[(b * MT + r) * kc + c] = a.y[(2 * (t0 + b)) * mk + r * k + c0 + c];
    }
    __syncthreads();

    for (int e = tid; e < nbh * kw; e += NT) {
        const int b = e / kw, c = e - b * kw;
        trsv_lower_col<MT>(sL + b * MT * MT, sInv + b * MT, sR + b * MT * kc + c, kc, m);
    }
    __syncthreads();

    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        a.r[(t0 + b) * mk + r * k + c0 + c] = sR[(b * MT + r) * kc + c];
    }
    // Z^H r: rows p < m give P^H r (left even block), rows p >= m give Q^H r (right)
    for (int e = tid; e < nbh * kw * m2; e += NT) {
        const int b = e / (kw * m2), rem = e - b * (kw * m2), c = rem / m2, p = rem - c * m2;
        const int64_t t = t0 + b, pos = 2 * t;
        if (p < m ? (pos == 0) : (pos + 1 >= a.Nl)) continue;
        const z2 *Zt = a.Z + t * (int64_t)(m * m2);
        const z2 *Rb = sR + b * MT * kc + c;
        z2 acc = zmk(0.0, 0.0);
#pragma unroll
        for (int s = 0; s < MT; ++s)
            if (s < m) zmac_ca(acc, __ldg(Zt + s * m2 + p), Rb[s * kc]);
        if (p < m) a.cl[t * mk + p * k + c0 + c] = acc;
        else a.cr[t * mk + (p - m) * k + c0 + c] = acc;
    }
}

__global__ void __launch_bounds__(256) k_solve_down_even(LevelArgs a) {
    const int64_t mk = (int64_t)a.m * a.k, total = a.ne * mk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / mk, rem = e - j * mk;
        z2 v = a.y[(2 * j + 1) * mk + rem];
        v = zsub(v, a.cr[j * mk + rem]);                          // Q^H r of odd block j (left)
        if (j + 1 < a.no) v = zsub(v, a.cl[(j + 1) * mk + rem]);  // P^H r of odd block j+1 (right)
        a.yn[j * mk + rem] = v;
    }
}

// --------------------------------------------------------------- solve: up

template <int MT>
__global__ void __launch_bounds__(256) k_solve_up(LevelArgs a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int m = a.m, k = a.k, nb = a.nb, kc = a.kc, NT = blockDim.x, tid = threadIdx.x;
    const int mm = m * m, m2 = 2 * m, mk = m * k;
    const int c0 = blockIdx.y * kc, kw = min(kc, k - c0);
    const int64_t t0 = (int64_t)blockIdx.x * nb;
    const int nbh = (int)min((int64_t)nb, a.no - t0);
    z2 *sL = reinterpret_cast<z2 *>(smem_raw);                                // [nb][MT][MT]
    z2 *sW = sL + (size_t)nb * MT * MT;                                        // [nb][MT][kc]
    z2 *sX = sW + (size_t)nb * MT * kc;                                        // [nb][2MT][kc]
    double *sInv = reinterpret_cast<double *>(sX + (size_t)nb * 2 * MT * kc);  // [nb][MT]

    if (a.level == 0 && *a.status != CRS_NO_FAIL) {
        // the factorisation broke down: the result is NaN
        const z2 nan2 = zmk(__longlong_as_double(0x7ff8000000000000ll), __longlong_as_double(0x7ff8000000000000ll));
        for (int e = tid; e < nbh * m * kw; e += NT) {
            const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
            const int64_t t = t0 + b;
            a.x[(2 * t) * mk + r * k + c0 + c] = nan2;
            if (t < a.ne) a.x[(2 * t + 1) * mk + r * k + c0 + c] = nan2;
        }
        return;
    }

    for (int e = tid; e < nbh * mm; e += NT) {
        const int b = e / mm, rem = e - b * mm, r = rem / m, c = rem - r * m;
        sL[(b * MT + r) * MT + c] = a.L[(t0 + b) * mm + rem];
    }
    for (int e = tid; e < nbh * m; e += NT) {
        const int b = e / m, r = e - b * m;
        sInv[b * MT + r] = a.inv[(t0 + b) * m + r];
    }
    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        const int64_t t = t0 + b;
        sW[(b * MT + r) * kc + c] = a.r[t * mk + r * k + c0 + c];
        // [x_left; x_right] = [xn_{t-1}; xn_t], zero past the boundary
        sX[(b * 2 * MT + r) * kc + c] = (t >= 1) ? a.xn[(t - 1) * mk + r * k + c0 + c] : zmk(0.0, 0.0);
        const z2 xr = (t < a.ne) ? a.xn[t * mk + r * k + c0 + c] : zmk(0.0, 0.0);
        sX[(b * 2 * MT + m + r) * kc + c] = xr;
        if (t < a.ne) a.x[(2 * t + 1) * mk + r * k + c0 + c] = xr;  // even unknowns
    }
    __syncthreads();

    // w = r - P x_left - Q x_right
    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        const int64_t t = t0 + b;
        const z2 *Zr = a.Z + t * (int64_t)(m * m2) + r * m2;
        const z2 *Xb = sX + b * 2 * MT * kc + c;
        z2 acc = sW[(b * MT + r) * kc + c];
#pragma unroll
        for (int s = 0; s < 2 * MT; ++s)
            if (s < m2) zmsub(acc, __ldg(Zr + s), Xb[s * kc]);
        sW[(b * MT + r) * kc + c] = acc;
    }
    __syncthreads();

    // x_odd = L^{-H} w
    for (int e = tid; e < nbh * kw; e += NT) {
        const int b = e / kw, c = e - b * kw;
        trsv_lower_h_col<MT>(sL + b * MT * MT, sInv + b * MT, sW + b * MT * kc + c, kc, m);
    }
    __syncthreads();
    for (int e = tid; e < nbh * m * kw; e += NT) {
        const int b = e / (m * kw), rem = e - b * (m * kw), r = rem / kw, c = rem - r * kw;
        a.x[(2 * (t0 + b)) * mk + r * k + c0 + c] = sW[(b * MT + r) * kc + c];
    }
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

TileShape tile_shape(int mt) {
    switch (mt) {
        case 4: return {32, 32, 32, 256};
        case 8: return {16, 16, 16, 256};
        case 16: return {4, 8, 16, 256};
        case 32: return {2, 2, 32, 256};
        case 64: return {1, 1, 32, 256};
        default: return {0, 0, 0, 0};
    }
}

int pick_mt(int m) {
    if (m <= 4) return 4;
    if (m <= 8) return 8;
    if (m <= 16) return 16;
    if (m <= 32) return 32;
    if (m <= 64) return 64;
    return 0;
}

size_t factor_smem_bytes(int mt, int nb) {
    return (size_t)nb * (3 * (size_t)mt * mt * sizeof(z2) + (size_t)mt * sizeof(double));
}

size_t solve_smem_bytes(int mt, int nb, int kc, bool up) {
    return (size_t)nb * ((size_t)mt * mt * sizeof(z2) + (size_t)mt * kc * sizeof(z2) * (up ? 3 : 1) +
                         (size_t)mt * sizeof(double));
}

template <int MT>
static cudaError_t prepare_mt() {
    const TileShape ts = tile_shape(MT);
    cudaError_t e;
    e = cudaFuncSetAttribute(k_factor_odd<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)factor_smem_bytes(MT, ts.nb_factor));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_solve_down_odd<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)solve_smem_bytes(MT, ts.nb_solve, ts.kc_max, false));
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(k_solve_up<MT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)solve_smem_bytes(MT, ts.nb_solve, ts.kc_max, true));
}

cudaError_t prepare_kernels(int mt) {
    switch (mt) {
        case 4: return prepare_mt<4>();
        case 8: return prepare_mt<8>();
        case 16: return prepare_mt<16>();
        case 32: return prepare_mt<32>();
        case 64: return prepare_mt<64>();
        default: return cudaErrorInvalidValue;
    }
}

// Odd blocks per CTA for a level with `no` odd blocks: the tile's maximum,
// shrunk on small levels so that about two CTAs land on every SM.
static int level_nb(int nb_max, int64_t no, int nsm) {
    int64_t want = (no + 2 * (int64_t)nsm - 1) / (2 * (int64_t)nsm);
    if (want < 1) want = 1;
    return (int)(want < nb_max ? want : nb_max);
}

static unsigned grid_1d(int64_t items, int nsm) {
    int64_t g = (items + 255) / 256;
    const int64_t cap = (int64_t)nsm * 16;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return (unsigned)g;
}

template <int MT>
static cudaError_t factor_odd_mt(LevelArgs a, int nsm, cudaStream_t s) {
    const TileShape ts = tile_shape(MT);
    a.nb = level_nb(ts.nb_factor, a.no, nsm);
    const unsigned grid = (unsigned)((a.no + a.nb - 1) / a.nb);
    k_factor_odd<MT><<<grid, ts.threads, factor_smem_bytes(MT, a.nb), s>>>(a);
    return cudaGetLastError();
}

template <int MT>
static cudaError_t solve_down_odd_mt(LevelArgs a, int nsm, cudaStream_t s) {
    const TileShape ts = tile_shape(MT);
    a.nb = level_nb(ts.nb_solve, a.no, nsm);
    a.kc = a.k < ts.kc_max ? a.k : ts.kc_max;
    const dim3 grid((unsigned)((a.no + a.nb - 1) / a.nb), (unsigned)((a.k + a.kc - 1) / a.kc));
    k_solve_down_odd<MT><<<grid, ts.threads, solve_smem_bytes(MT, a.nb, a.kc, false), s>>>(a);
    return cudaGetLastError();
}

template <int MT>
static cudaError_t solve_up_mt(LevelArgs a, int nsm, cudaStream_t s) {
    const TileShape ts = tile_shape(MT);
    a.nb = level_nb(ts.nb_solve, a.no, nsm);
    a.kc = a.k < ts.kc_max ? a.k : ts.kc_max;
    const dim3 grid((unsigned)((a.no + a.nb - 1) / a.nb), (unsigned)((a.k + a.kc - 1) / a.kc));
    k_solve_up<MT><<<grid, ts.threads, solve_smem_bytes(MT, a.nb, a.kc, true), s>>>(a);
    return cudaGetLastError();
}

#define CRS_DISPATCH(fn, mt, ...)                   \
    switch (mt) {                                   \
        case 4: return fn<4>(__VA_ARGS__);          \
        case 8: return fn<8>(__VA_ARGS__);          \
        case 16: return fn<16>(__VA_ARGS__);        \
        case 32: return fn<32>(__VA_ARGS__);        \
        case 64: return fn<64>(__VA_ARGS__);        \
        default: return cudaErrorInvalidValue;      \
    }

cudaError_t launch_factor_odd(int mt, const LevelArgs &a, int nsm, cudaStream_t s) {
    CRS_DISPATCH(factor_odd_mt, mt, a, nsm, s)
}
cudaError_t launch_factor_even(const LevelArgs &a, int nsm, cudaStream_t s) {
    if (a.ne == 0) return cudaSuccess;
    k_factor_even<<<grid_1d(a.ne * (a.m * (a.m + 1) / 2), nsm), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_solve_down_odd(int mt, const LevelArgs &a, int nsm, cudaStream_t s) {
    CRS_DISPATCH(solve_down_odd_mt, mt, a, nsm, s)
}
cudaError_t launch_solve_down_even(const LevelArgs &a, int nsm, cudaStream_t s) {
    if (a.ne == 0) return cudaSuccess;
    k_solve_down_even<<<grid_1d(a.ne * a.m * a.k, nsm), 256, 0, s>>>(a);
    return cudaGetLastError();
}
cudaError_t launch_solve_up_level(int mt, const LevelArgs &a, int nsm, cudaStream_t s) {
    CRS_DISPATCH(solve_up_mt, mt, a, nsm, s)
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
