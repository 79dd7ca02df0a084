// cr_alg1.cu -- the two small kernels of the Algorithm 1 driver (the reduction
// levels themselves run the classic level kernels, see crsolve_api.cu).
//
// Layout.  A level of Algorithm 1 (Sec. 3) holds 2^l independent split
// systems of n = N/2^l blocks, stored one after another as one concatenated
// block-tridiagonal system of N blocks whose couplings across system
// boundaries are zero.  Each level buffer keeps one auxiliary block in front
// of the concatenation: A[0] = I, B[0] = 0, y[0] = 0 (the paper's boundary
// auxiliaries A_0 = I, B_0 = 0), so that the same buffer, read from block 1,
// is the concatenation itself, and, read from block 0, the concatenation
// shifted by one, whose even half is the odd half of every split system.
#include "cr_launch.h"

namespace crs {

namespace {

__global__ void k_alg1_border(z2 *A0, z2 *A1, z2 *B0, z2 *B1, z2 *B1mid, int m) {
    const int mm = m * m;
    for (int e = threadIdx.x; e < mm; e += blockDim.x) {
        const int r = e / m, c = e - r * m;
        const z2 one = make_double2(r == c ? 1.0 : 0.0, 0.0), zero = make_double2(0.0, 0.0);
        A0[e] = one;
        A1[e] = one;
        if (B0) B0[e] = zero;
        if (B1) B1[e] = zero;
        if (B1mid) B1mid[e] = zero;
    }
}

// x [N][mk] already holds the blocks at even concatenated positions (the
// reduction that starts at block 1); the odd ones come from xb [N+1][mk] (the
// shifted reduction), one block further on.  After a breakdown: NaN.
__global__ void k_alg1_merge(z2 *x, const z2 *xb, int64_t N, int64_t mk, const unsigned long long *status) {
    const bool failed = *status != CRS_NO_FAIL;
    const z2 nan2 = make_double2(qnan(0.0), qnan(0.0));
    const int64_t n = N * mk, stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += stride) {
        if (failed) x[e] = nan2;
        else if ((e / mk) & 1) x[e] = xb[e + mk];
    }
}

}  // namespace

cudaError_t launch_alg1_border(z2 *A0, z2 *A1, z2 *B0, z2 *B1, z2 *B1mid, int m, cudaStream_t s) {
    k_alg1_border<<<1, 256, 0, s>>>(A0, A1, B0, B1, B1mid, m);
    return cudaGetLastError();
}

cudaError_t launch_alg1_merge(z2 *x, const z2 *xb, int64_t N, int64_t mk, const unsigned long long *status,
                              int nsm, cudaStream_t s) {
    const int64_t n = N * mk;
    const int64_t want = (n + 255) / 256;
    const int grid = (int)(want < (int64_t)nsm * 4 ? (want > 0 ? want : 1) : (int64_t)nsm * 4);
    k_alg1_merge<<<grid, 256, 0, s>>>(x, xb, N, mk, status);
    return cudaGetLastError();
}

}  // namespace crs
