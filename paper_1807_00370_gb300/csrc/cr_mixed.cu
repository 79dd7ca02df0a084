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

cudaError_t launch_residual(int64_t N, int m, int k, const z2 *A, const z2 *B, const z2 *x, const z2 *y, z2 *r,
                            int nsm, cudaStream_t s) {
    k_residual<<<grid_for(N * m * k, nsm * 8), 256, 0, s>>>(N, m, k, A, B, x, y, r);
    return cudaGetLastError();
}

}  // namespace crs
