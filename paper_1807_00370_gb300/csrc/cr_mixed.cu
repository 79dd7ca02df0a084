// cr_mixed.cu -- kernels of the mixed-precision form: the fine reduction
// levels run in FP32 (the same level kernels, instantiated for float), the
// coarsest levels, the residual and the iterative refinement in FP64.
//
//   k_convert         complex FP64 <-> FP32 copies between the two halves
//   k_update          x += d (d from the FP32 correction solve, accumulated in
//                     FP64) and the infinity norms of d and the new x
//   k_residual        r = y - A x in FP64 for the block-tridiagonal A of
//                     eq. Axb (A_j Hermitian from its lower triangle)
#include "cr_launch.h"

namespace crs {

template <class Cin, class Cout>
__global__ void __launch_bounds__(256) k_convert(const Cin *__restrict__ in, Cout *__restrict__ out, int64_t n) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const Cin v = in[e];
        Cout w;
        w.x = v.x;
        w.y = v.y;
        out[e] = w;
    }
}

// Non-negative doubles order like their bit patterns, so atomicMax on the
// bits is a max on the values.
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long *slot, double v) {
    atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

__global__ void __launch_bounds__(256) k_update(z2 *__restrict__ x, const c2 *__restrict__ d, int64_t n, int first,
                                                unsigned long long *norms /* [2]: |d|_inf, |x|_inf */) {
    double dmax = 0.0, xmax = 0.0;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const c2 dv = d[e];
        z2 xv = first ? zmk(0.0, 0.0) : x[e];
        xv.x += (double)dv.x;
        xv.y += (double)dv.y;
        x[e] = xv;
        dmax = fmax(dmax, fmax(fabs((double)dv.x), fabs((double)dv.y)));
        xmax = fmax(xmax, fmax(fabs(xv.x), fabs(xv.y)));
    }
    for (int o = 16; o > 0; o >>= 1) {
        dmax = fmax(dmax, __shfl_xor_sync(0xffffffffu, dmax, o));
        xmax = fmax(xmax, __shfl_xor_sync(0xffffffffu, xmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        atomic_max_nonneg(norms, dmax);
        atomic_max_nonneg(norms + 1, xmax);
    }
}

// r_j = y_j - A_j x_j - B_{j-1} x_{j-1} - B_j^H x_{j+1}; one thread per entry
// (j, a, c), three dot products of length m in FP64.  The Hermitian A_j is
// read from its lower triangle in three loops (s < a, s = a, s > a) and the
// conjugations are folded into the FMAs, so each term is exactly 4 DFMA.
__global__ void __launch_bounds__(256) k_residual(int64_t N, int m, int k, const z2 *__restrict__ A,
                                                  const z2 *__restrict__ B, const z2 *__restrict__ x,
                                                  const z2 *__restrict__ y, z2 *__restrict__ r) {
    const int64_t mk = (int64_t)m * k, mm = (int64_t)m * m, total = N * mk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t j = e / mk;
        const int rem = (int)(e - j * mk), a = rem / k, c = rem - a * k;
        z2 acc = y[e];
        const z2 *Aj = A + j * mm, *xj = x + j * mk + c;
        for (int s = 0; s < a; ++s) zmsub(acc, __ldg(Aj + a * m + s), __ldg(xj + (int64_t)s * k));
        {
            const double d = __ldg(&Aj[a * m + a].x);
            const z2 xv = __ldg(xj + (int64_t)a * k);
            acc.x = fma(-d, xv.x, acc.x);
            acc.y = fma(-d, xv.y, acc.y);
        }
        for (int s = a + 1; s < m; ++s) zmsub_ca(acc, __ldg(Aj + s * m + a), __ldg(xj + (int64_t)s * k));
        if (j >= 1) {
            const z2 *Bl = B + (j - 1) * mm + a * m, *xl = x + (j - 1) * mk + c;
            for (int s = 0; s < m; ++s) zmsub(acc, __ldg(Bl + s), __ldg(xl + (int64_t)s * k));
        }
        if (j + 1 < N) {
            const z2 *Br = B + j * mm + a, *xr = x + (j + 1) * mk + c;
            for (int s = 0; s < m; ++s) zmsub_ca(acc, __ldg(Br + (int64_t)s * m), __ldg(xr + (int64_t)s * k));
        }
        r[e] = acc;
    }
}

// ---------------------------------------------------------------- PCG
//
// Per right-hand-side column c (k independent conjugate-gradient runs on the
// n = N m rows of the block vectors): dot products Re sum conj(a) b, the
// update x += alpha p, r += alpha w (w = -A p) with the per-column maxima of
// |alpha p| and |x|, and the direction p = z + beta p.  A dot product is
// reduced in a fixed order (per-thread sums, a shared-memory tree, then the
// CTA partials in CTA order), so it is the same from run to run.

constexpr int kDotThreads = 256;

template <class CB>
__global__ void __launch_bounds__(kDotThreads) k_dot_partial(const z2 *__restrict__ a, const CB *__restrict__ b,
                                                             int64_t rows, int k, int kc0, double *__restrict__ part) {
    // columns kc0 .. kc0 + kw - 1 of this pass; tpc threads per column
    const int kw = min(k - kc0, kDotThreads), tpc = kDotThreads / kw;
    const int tid = threadIdx.x, c = tid % kw, lane_r = tid / kw;
    double sum = 0.0;
    if (lane_r < tpc) {
        const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
        const int64_t r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
        for (int64_t r = r0 + lane_r; r < r1; r += tpc) {
            const z2 av = a[r * k + kc0 + c];
            const CB bv = b[r * k + kc0 + c];
            sum = fma(av.x, (double)bv.x, sum);
            sum = fma(av.y, (double)bv.y, sum);
        }
    }
    __shared__ double red[kDotThreads];
    red[tid] = sum;
    __syncthreads();
    if (tid < kw) {
        double t = 0.0;
        for (int q = 0; q < tpc; ++q) t += red[q * kw + tid];
        part[(int64_t)blockIdx.x * k + kc0 + tid] = t;
    }
}

// out[c] = sum over CTAs of part[g][c] in CTA order; mode 0: out = the dot,
// mode 1: alpha[c] = num[c] / (-dot) (dot = (p, w) = -(p, A p)), a non-positive
// or non-finite curvature sets *flag; mode 2: beta[c] = (dot - num2[c]) /
// num[c] and num[c] = dot (flexible Polak-Ribiere, num = the previous (r, z)).
__global__ void k_dot_finish(const double *__restrict__ part, int G, int k, double *out, int mode, double *num,
                             const double *num2, int *flag) {
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < k; c += gridDim.x * blockDim.x) {
        double t = 0.0;
        for (int g = 0; g < G; ++g) t += part[(int64_t)g * k + c];
        if (mode == 0) {
            out[c] = t;
        } else if (mode == 1) {
            const double pAp = -t;
            if (!(pAp > 0.0) || !(num[c] == num[c])) {
                out[c] = 0.0;
                if (flag) *flag = 1;
            } else {
                out[c] = num[c] / pAp;
            }
        } else {
            const double b = num[c] != 0.0 ? (t - num2[c]) / num[c] : 0.0;
            out[c] = b == b ? b : 0.0;
            num[c] = t;
        }
    }
}

// Threads are laid out like k_dot_partial (a column per thread, a row range
// per CTA), so each thread keeps the maxima of one column and a CTA does one
// atomic per column.
__global__ void __launch_bounds__(kDotThreads) k_pcg_update(z2 *__restrict__ x, z2 *__restrict__ r,
                                                            const z2 *__restrict__ p, const z2 *__restrict__ w,
                                                            const double *__restrict__ alpha, int64_t rows, int k,
                                                            int kc0, unsigned long long *norms /* [2k] */) {
    const int kw = min(k - kc0, kDotThreads), tpc = kDotThreads / kw;
    const int tid = threadIdx.x, c = tid % kw, lane_r = tid / kw;
    double dmax = 0.0, xmax = 0.0;
    if (lane_r < tpc) {
        const double al = alpha[kc0 + c];
        const int64_t per = (rows + gridDim.x - 1) / gridDim.x;
        const int64_t r0 = blockIdx.x * per, r1 = min(rows, r0 + per);
        for (int64_t rr = r0 + lane_r; rr < r1; rr += tpc) {
            const int64_t e = rr * k + kc0 + c;
            const z2 pv = p[e], wv = w[e];
            z2 xv = x[e], rv = r[e];
            const double dx = al * pv.x, dy = al * pv.y;
            xv.x += dx;
            xv.y += dy;
            rv.x = fma(al, wv.x, rv.x);
            rv.y = fma(al, wv.y, rv.y);
            x[e] = xv;
            r[e] = rv;
            dmax = fmax(dmax, fmax(fabs(dx), fabs(dy)));
            xmax = fmax(xmax, fmax(fabs(xv.x), fabs(xv.y)));
        }
    }
    __shared__ double sd[kDotThreads], sx[kDotThreads];
    sd[tid] = dmax;
    sx[tid] = xmax;
    __syncthreads();
    if (tid < kw) {
        for (int q = 1; q < tpc; ++q) {
            dmax = fmax(dmax, sd[q * kw + tid]);
            xmax = fmax(xmax, sx[q * kw + tid]);
        }
        atomic_max_nonneg(norms + kc0 + tid, dmax);
        atomic_max_nonneg(norms + k + kc0 + tid, xmax);
    }
}

__global__ void __launch_bounds__(256) k_pcg_direction(z2 *__restrict__ p, const c2 *__restrict__ z,
                                                       const double *__restrict__ beta, int64_t n, int k, int first) {
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const c2 zv = z[e];
        z2 pv = first ? zmk(0.0, 0.0) : p[e];
        const double b = first ? 0.0 : beta[(int)(e % k)];
        pv.x = fma(b, pv.x, (double)zv.x);
        pv.y = fma(b, pv.y, (double)zv.y);
        p[e] = pv;
    }
}

static unsigned grid_for(int64_t items, int nsm) {
    int64_t g = (items + 255) / 256;
    const int64_t cap = (int64_t)nsm * 16;
    return (unsigned)(g > cap ? cap : (g < 1 ? 1 : g));
}

cudaError_t launch_to_f32(const z2 *in, c2 *out, int64_t n, int nsm, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_convert<z2, c2><<<grid_for(n, nsm), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_to_f64(const c2 *in, z2 *out, int64_t n, int nsm, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    k_convert<c2, z2><<<grid_for(n, nsm), 256, 0, s>>>(in, out, n);
    return cudaGetLastError();
}

cudaError_t launch_update(z2 *x, const c2 *d, int64_t n, int first, unsigned long long *norms, int nsm,
                          cudaStream_t s) {
    k_update<<<grid_for(n, nsm), 256, 0, s>>>(x, d, n, first, norms);
    return cudaGetLastError();
}

int dot_partials(int nsm) { return 4 * nsm; }

template <class CB>
static cudaError_t launch_dot_t(const z2 *a, const CB *b, int64_t rows, int k, double *part, double *out, int mode,
                                double *num, const double *num2, int *flag, int nsm, cudaStream_t s) {
    const int G = dot_partials(nsm);
    for (int kc0 = 0; kc0 < k; kc0 += kDotThreads) {
        k_dot_partial<CB><<<G, kDotThreads, 0, s>>>(a, b, rows, k, kc0, part);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_dot_finish<<<(k + 127) / 128, 128, 0, s>>>(part, G, k, out, mode, num, num2, flag);
    return cudaGetLastError();
}

cudaError_t launch_dot(const z2 *a, const c2 *b, int64_t rows, int k, double *part, double *out, int mode, double *num,
                       const double *num2, int *flag, int nsm, cudaStream_t s) {
    return launch_dot_t(a, b, rows, k, part, out, mode, num, num2, flag, nsm, s);
}

cudaError_t launch_dot(const z2 *a, const z2 *b, int64_t rows, int k, double *part, double *out, int mode, double *num,
                       const double *num2, int *flag, int nsm, cudaStream_t s) {
    return launch_dot_t(a, b, rows, k, part, out, mode, num, num2, flag, nsm, s);
}

cudaError_t launch_pcg_update(z2 *x, z2 *r, const z2 *p, const z2 *w, const double *alpha, int64_t n, int k,
                              unsigned long long *norms, int nsm, cudaStream_t s) {
    const int64_t rows = n / k;
    for (int kc0 = 0; kc0 < k; kc0 += kDotThreads) {
        k_pcg_update<<<4 * nsm, kDotThreads, 0, s>>>(x, r, p, w, alpha, rows, k, kc0, norms);
        const cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t launch_pcg_direction(z2 *p, const c2 *z, const double *beta, int64_t n, int k, int first, int nsm,
                                 cudaStream_t s) {
    k_pcg_direction<<<grid_for(n, nsm), 256, 0, s>>>(p, z, beta, n, k, first);
    return cudaGetLastError();
}

cudaError_t launch_residual(int64_t N, int m, int k, const z2 *A, const z2 *B, const z2 *x, const z2 *y, z2 *r,
                            int nsm, cudaStream_t s) {
    k_residual<<<grid_for(N * m * k, nsm * 8), 256, 0, s>>>(N, m, k, A, B, x, y, r);
    return cudaGetLastError();
}

}  // namespace crs
