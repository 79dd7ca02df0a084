// cr_launch.h -- host-side launchers of the per-level kernels (internal).
#pragma once
#include <cuda_runtime.h>
#include "cr_device.cuh"

namespace crs {

// Per-MT tile shape: odd blocks per CTA for the factor and solve kernels and
// the widest right-hand-side chunk one solve CTA stages in shared memory.
struct TileShape {
    int nb_factor;
    int nb_solve;
    int kc_max;
    int threads;
};

TileShape tile_shape(int mt);
int pick_mt(int m);                                  // 4, 8, 16, 32, 64 or 0
size_t factor_smem_bytes(int mt, int nb);
size_t solve_smem_bytes(int mt, int nb, int kc, bool up);
cudaError_t prepare_kernels(int mt);                 // raise shared-memory limits once per device

// Factor sweep of one level: the odd-block kernel (Cholesky, P, Q, Z^H Z),
// then the even-block kernel (the next level's diagonal blocks).
cudaError_t launch_factor_odd(int mt, const LevelArgs &a, int nsm, cudaStream_t s);
cudaError_t launch_factor_even(const LevelArgs &a, int nsm, cudaStream_t s);
// Down sweep of one level: r and Z^H r on the odd blocks, then the next
// level's right-hand side on the even blocks.
cudaError_t launch_solve_down_odd(int mt, const LevelArgs &a, int nsm, cudaStream_t s);
cudaError_t launch_solve_down_even(const LevelArgs &a, int nsm, cudaStream_t s);
// Up sweep of one level (x of this level from the next level's x).
cudaError_t launch_solve_up_level(int mt, const LevelArgs &a, int nsm, cudaStream_t s);
// Adjoint outer products gA, gB from x and gy.
cudaError_t launch_adjoint_outer(int64_t N, int m, int k, const z2 *x, const z2 *gy, z2 *gA,
                                 z2 *gB, int nsm, cudaStream_t s);
// Fill n complex values with NaN if *status records a breakdown.
cudaError_t launch_nan_if_failed(z2 *x, int64_t n, const unsigned long long *status, int nsm,
                                 cudaStream_t s);

}  // namespace crs
