// cr_launch.h -- host-side launchers of the per-level kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include "cr_core.cuh"

namespace crs {

// Per-MT tile shape: odd blocks per CTA for the factor and solve kernels and
// the widest right-hand-side chunk one solve CTA stages in shared memory.
struct TileShape {
    int nb_factor;
    int nb_solve;
    int kc_max;
    int threads;        // threads per CTA of the factor kernels
    int threads_solve;  // threads per CTA of the solve kernels
};

TileShape tile_shape(int mt);
bool set_tile_shape(int mt, const TileShape &ts, size_t smem_limit);
bool set_tile_shape32(int mt, const TileShape &ts, size_t smem_limit);
int pick_mt(int m);                                  // 4, 8, 16, 32, 64 or 0
size_t factor_smem_bytes(int mt, int nb, int rsize = 8);           // rsize: 8 FP64, 4 FP32
size_t solve_smem_bytes(int mt, int nb, int kc, int panels, int rsize = 8);
cudaError_t prepare_kernels(int mt);                 // raise shared-memory limits once per device

// Odd blocks per CTA of a level with `no` odd blocks (the tile's maximum,
// shrunk on small levels so that about two CTAs land on every SM), and the
// right-hand-side chunk width of the solve kernels.
int factor_nb(int mt, int64_t no, int nsm);
int solve_nb(int mt, int64_t no, int nsm);
int solve_kc(int mt, int k, int64_t no, int nsm);
// the same for the FP32 levels of the mixed-precision form
TileShape tile_shape32(int mt);
int factor_nb32(int mt, int64_t no, int nsm);
int solve_nb32(int mt, int64_t no, int nsm);
int solve_kc32(int mt, int k, int64_t no, int nsm);
inline int64_t num_ctas(int64_t no, int nb) { return crs_num_ctas(no, nb); }

// Factor sweep of one level (a.nb set by factor_nb): the odd-block kernel
// (Cholesky, P, Q, Z^H Z, and the even blocks that lie inside its CTA), then
// the fix-up of the even blocks on CTA boundaries.  FP64 and FP32 versions.
cudaError_t launch_factor_odd(int mt, const LevelArgsT<double> &a, cudaStream_t s);
cudaError_t launch_factor_odd(int mt, const LevelArgsT<float> &a, cudaStream_t s);
cudaError_t launch_factor_fix(const LevelArgsT<double> &a, int nsm, cudaStream_t s);
cudaError_t launch_factor_fix(const LevelArgsT<float> &a, int nsm, cudaStream_t s);
// Down sweep of one level (a.nb, a.kc set): r, Z^H r and the next level's
// right-hand side inside each CTA, then the CTA-boundary fix-up.
cudaError_t launch_solve_down_odd(int mt, const LevelArgsT<double> &a, cudaStream_t s);
cudaError_t launch_solve_down_odd(int mt, const LevelArgsT<float> &a, cudaStream_t s);
cudaError_t launch_solve_down_fix(const LevelArgsT<double> &a, int nsm, cudaStream_t s);
cudaError_t launch_solve_down_fix(const LevelArgsT<float> &a, int nsm, cudaStream_t s);
// Up sweep of one level (x of this level from the next level's x).
cudaError_t launch_solve_up(int mt, const LevelArgsT<double> &a, cudaStream_t s);
cudaError_t launch_solve_up(int mt, const LevelArgsT<float> &a, cudaStream_t s);
// FP32 levels of class MT = 64 (cr_solve32.cu): the factor keeps L^{-1} in
// place of L and both sweeps run as complex products in persistent CTAs, one
// odd block and a.kc columns per work item (a.nb = 1; a.kc = 8, 16 or 32:
// solve_kc_g32(a.k), narrowed by solve_kc32 on levels with few odd blocks);
// launch_solve_down_odd / launch_solve_up route there.
int solve_kc_g32(int k);
cudaError_t prepare_solve_g32(int smem_optin);
cudaError_t launch_solve_down_g32(const LevelArgsT<float> &a, cudaStream_t s);
cudaError_t launch_solve_up_g32(const LevelArgsT<float> &a, cudaStream_t s);
// Mixed-precision helpers (cr_mixed.cu).
cudaError_t launch_to_f32(const z2 *in, c2 *out, int64_t n, int nsm, cudaStream_t s);
cudaError_t launch_to_f64(const c2 *in, z2 *out, int64_t n, int nsm, cudaStream_t s);
cudaError_t launch_update(z2 *x, const c2 *d, int64_t n, int first, unsigned long long *norms, int nsm,
                          cudaStream_t s);
cudaError_t launch_residual(int64_t N, int m, int k, const z2 *A, const z2 *B, const z2 *x, const z2 *y, z2 *r,
                            int nsm, cudaStream_t s);
// Preconditioned conjugate gradients of the mixed-precision form, per
// right-hand-side column (cr_mixed.cu).  launch_dot reduces Re sum conj(a) b
// over the rows = N m rows of [rows][k] block vectors into dot_partials(nsm)
// x k partial sums `part`, then (mode 0) out = the dots, (mode 1) out = alpha
// = num / (-dot) with *flag set on a non-positive curvature, or (mode 2) out =
// beta = (dot - num2) / num and num = dot.
int dot_partials(int nsm);
cudaError_t launch_dot(const z2 *a, const c2 *b, int64_t rows, int k, double *part, double *out, int mode, double *num,
                       const double *num2, int *flag, int nsm, cudaStream_t s);
cudaError_t launch_dot(const z2 *a, const z2 *b, int64_t rows, int k, double *part, double *out, int mode, double *num,
                       const double *num2, int *flag, int nsm, cudaStream_t s);
// x += alpha p, r += alpha w over n = N m k entries; norms[c] = max |alpha p|,
// norms[k + c] = max |x| of column c (atomic max, zeroed by the caller).
cudaError_t launch_pcg_update(z2 *x, z2 *r, const z2 *p, const z2 *w, const double *alpha, int64_t n, int k,
                              unsigned long long *norms, int nsm, cudaStream_t s);
// p = z + beta p (first: p = z); z is the FP32 correction.
cudaError_t launch_pcg_direction(z2 *p, const c2 *z, const double *beta, int64_t n, int k, int first, int nsm,
                                 cudaStream_t s);
// FP64 residual r = y - A x by exact splitting on the BF16 tensor cores
// (cr_resid_tc.cu, m <= 64).  erow [N][m] holds the binary exponent of the
// largest entry of every row of [B_{j-1} | A_j | B_j^H] (launch_row_exponents,
// once per matrix); ecol [N][k] the largest exponent of every column of every
// x_j (computed by launch_residual_tc before the product).
struct ResidTcArgs {
    int64_t N;
    int m, k;
    const z2 *A, *B, *x, *y;   // y may be NULL (r = -A x)
    z2 *r;
    int *erow, *ecol;
    int *err;      // set to 1 if a bounded wait gave up
    unsigned long long *dbg;   // bounds-checked builds: first out-of-range access
    // optional: the matrix slices of every (block row, K-chunk) precomputed in
    // the shared-memory layout (residual_image_bytes(N), launch_matrix_image);
    // the product then copies them in instead of cutting the matrix each time
    const unsigned char *img;
};
size_t residual_tc_smem_bytes();
size_t residual_image_bytes(int64_t N);
cudaError_t launch_row_exponents(const ResidTcArgs &a, int nsm, cudaStream_t s);
cudaError_t launch_matrix_image(const ResidTcArgs &a, unsigned char *img, int nsm, cudaStream_t s);
cudaError_t launch_residual_tc(const ResidTcArgs &a, int nsm, cudaStream_t s);
// Adjoint outer products gA, gB from x and gy.
cudaError_t launch_adjoint_outer(int64_t N, int m, int k, const z2 *x, const z2 *gy, z2 *gA,
                                 z2 *gB, int nsm, cudaStream_t s);
// Algorithm 1 driver: the fixed border blocks of the two level buffers
// (A0[0] = A1[0] = I; B0, B1, B1mid = 0 where non-null), and the final merge of
// the two base reductions' solutions (NaN after a breakdown).
cudaError_t launch_alg1_border(z2 *A0, z2 *A1, z2 *B0, z2 *B1, z2 *B1mid, int m, cudaStream_t s);
cudaError_t launch_alg1_merge(z2 *x, const z2 *xb, int64_t N, int64_t mk, const unsigned long long *status,
                              int nsm, cudaStream_t s);
// Fill n complex values with NaN if *status records a breakdown.
cudaError_t launch_nan_if_failed(z2 *x, int64_t n, const unsigned long long *status, int nsm,
                                 cudaStream_t s);

}  // namespace crs
