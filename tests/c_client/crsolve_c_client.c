/*
 * A plain C client of libcrsolve.so: no Python, no torch.  It allocates
 * device memory with the CUDA runtime, drives the C ABI declared in
 * include/crsolve.h (plan, workspace, factor, solve, info, host-buffer solve,
 * error codes) and checks the solution against the definition of the problem:
 * the residual y - A x of the block-tridiagonal system, computed here on the
 * host.  Test infrastructure, built and run by tests/test_gpu_c_client.py.
 *
 * Input: a seeded, diagonally dominant Hermitian system (xorshift64 numbers):
 * B_j entries uniform in [-0.5, 0.5]^2 / m, A_j = H_j + (m + 2) I with H_j a
 * Hermitian matrix of entries uniform in [-0.5, 0.5]^2, y uniform.
 * Exit status 0 when every check passes.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime.h>

#include "crsolve.h"

static uint64_t rng_state = 0x9E3779B97F4A7C15ull;
static double uni(void) { /* uniform in [-0.5, 0.5) */
    rng_state ^= rng_state << 13;
    rng_state ^= rng_state >> 7;
    rng_state ^= rng_state << 17;
    return (double)(rng_state >> 11) * (1.0 / 9007199254740992.0) - 0.5;
}

#define CHECK(cond, ...)                         \
    do {                                         \
        if (!(cond)) {                           \
            fprintf(stderr, "FAIL: " __VA_ARGS__); \
            fprintf(stderr, "\n");               \
            return 1;                            \
        }                                        \
    } while (0)

/* r = y - A x for the block-tridiagonal system (A Hermitian from its lower triangle) */
static double residual_eta(int64_t N, int m, int k, const crsolve_z *A, const crsolve_z *B, const crsolve_z *y,
                           const crsolve_z *x) {
    double rmax = 0.0, xmax = 0.0, amax = 0.0;
    for (int64_t j = 0; j < N; ++j)
        for (int r = 0; r < m; ++r) {
            double rowsum = 0.0;
            for (int c = 0; c < k; ++c) {
                double re = y[(j * m + r) * k + c].re, im = y[(j * m + r) * k + c].im;
                for (int q = 0; q < m; ++q) {
                    /* A_j[r][q] from the lower triangle (Hermitian), real diagonal */
                    crsolve_z a = r >= q ? A[(j * m + r) * m + q] : A[(j * m + q) * m + r];
                    if (r < q) a.im = -a.im;
                    if (r == q) a.im = 0.0;
                    const crsolve_z xv = x[(j * m + q) * k + c];
                    re -= a.re * xv.re - a.im * xv.im;
                    im -= a.re * xv.im + a.im * xv.re;
                    if (c == 0) rowsum += hypot(a.re, a.im);
                    if (j > 0) { /* B_{j-1} x_{j-1}: B_{j-1} sits at (j, j-1) */
                        const crsolve_z b = B[((j - 1) * m + r) * m + q], xl = x[((j - 1) * m + q) * k + c];
                        re -= b.re * xl.re - b.im * xl.im;
                        im -= b.re * xl.im + b.im * xl.re;
                        if (c == 0) rowsum += hypot(b.re, b.im);
                    }
                    if (j + 1 < N) { /* B_j^H x_{j+1} */
                        const crsolve_z b = B[(j * m + q) * m + r], xr = x[((j + 1) * m + q) * k + c];
                        re -= b.re * xr.re + b.im * xr.im;
                        im -= b.re * xr.im - b.im * xr.re;
                        if (c == 0) rowsum += hypot(b.re, b.im);
                    }
                }
                const double rv = hypot(re, im), xv = hypot(x[(j * m + r) * k + c].re, x[(j * m + r) * k + c].im);
                if (rv > rmax) rmax = rv;
                if (xv > xmax) xmax = xv;
            }
            if (rowsum > amax) amax = rowsum;
        }
    return rmax / (amax * xmax);
}

int main(int argc, char **argv) {
    const int64_t N = argc > 1 ? atoll(argv[1]) : 1000;
    const int m = argc > 2 ? atoi(argv[2]) : 8, k = argc > 3 ? atoi(argv[3]) : 3;
    const size_t nA = (size_t)N * m * m, nB = (size_t)(N - 1) * m * m, ny = (size_t)N * m * k;
    crsolve_z *A = calloc(nA, sizeof *A), *B = calloc(nB ? nB : 1, sizeof *B), *y = calloc(ny, sizeof *y);
    crsolve_z *x = calloc(ny, sizeof *x), *x2 = calloc(ny, sizeof *x2);
    CHECK(A && B && y && x && x2, "host allocation");
    for (size_t i = 0; i < nB; ++i) B[i] = (crsolve_z){uni() / m, uni() / m};
    for (int64_t j = 0; j < N; ++j)
        for (int r = 0; r < m; ++r)
            for (int q = 0; q <= r; ++q) {
                crsolve_z v = {uni(), r == q ? 0.0 : uni()};
                if (r == q) v.re += m + 2.0;
                A[(j * m + r) * m + q] = v;
                A[(j * m + q) * m + r] = (crsolve_z){v.re, -v.im};
            }
    for (size_t i = 0; i < ny; ++i) y[i] = (crsolve_z){uni(), uni()};

    crsolve_z *dA, *dB = NULL, *dy, *dx;
    CHECK(cudaMalloc((void **)&dA, nA * sizeof *dA) == cudaSuccess, "cudaMalloc A");
    if (N > 1) CHECK(cudaMalloc((void **)&dB, nB * sizeof *dB) == cudaSuccess, "cudaMalloc B");
    CHECK(cudaMalloc((void **)&dy, ny * sizeof *dy) == cudaSuccess, "cudaMalloc y");
    CHECK(cudaMalloc((void **)&dx, ny * sizeof *dx) == cudaSuccess, "cudaMalloc x");
    cudaMemcpy(dA, A, nA * sizeof *A, cudaMemcpyHostToDevice);
    if (N > 1) cudaMemcpy(dB, B, nB * sizeof *B, cudaMemcpyHostToDevice);
    cudaMemcpy(dy, y, ny * sizeof *y, cudaMemcpyHostToDevice);

    /* device path: plan, caller-owned workspace, factor, solve */
    crsolve_plan p = NULL;
    CHECK(crsolve_plan_create(N, m, k, CRSOLVE_FP64, 0, &p) == CRSOLVE_OK, "plan_create");
    size_t wsb = 0;
    CHECK(crsolve_workspace_bytes(p, &wsb) == CRSOLVE_OK, "workspace_bytes");
    void *ws = NULL;
    CHECK(cudaMalloc(&ws, wsb) == cudaSuccess, "cudaMalloc workspace");
    CHECK(crsolve_set_workspace(p, ws, wsb) == CRSOLVE_OK, "set_workspace");
    CHECK(crsolve_solve(p, k, dy, dx, NULL) == CRSOLVE_ENOTFACTORED, "solve before factor must be refused");
    CHECK(crsolve_factor(p, dA, dB, NULL) == CRSOLVE_OK, "factor");
    CHECK(crsolve_solve(p, k, dy, dx, NULL) == CRSOLVE_OK, "solve");
    CHECK(crsolve_solve(p, k, dy, dy, NULL) == CRSOLVE_EINVAL, "aliased x and y must be refused");
    crsolve_info info;
    CHECK(crsolve_info_get(p, &info, NULL) == CRSOLVE_OK && info.status == CRSOLVE_OK, "info");
    CHECK(cudaMemcpy(x, dx, ny * sizeof *x, cudaMemcpyDeviceToHost) == cudaSuccess, "copy x");
    const double eta = residual_eta(N, m, k, A, B, y, x);
    printf("device path: N=%lld m=%d k=%d residual eta %.3e\n", (long long)N, m, k, eta);
    CHECK(eta <= 1e-13, "residual %.3e", eta);

    /* host-buffer path: same result, bit for bit */
    crsolve_plan ph = NULL;
    CHECK(crsolve_plan_create(N, m, k, CRSOLVE_FP64, CRSOLVE_PLAN_HOST_STAGING, &ph) == CRSOLVE_OK, "plan_create host");
    size_t wsh = 0;
    crsolve_workspace_bytes(ph, &wsh);
    void *wsp = NULL;
    CHECK(cudaMalloc(&wsp, wsh) == cudaSuccess, "cudaMalloc host-plan workspace");
    CHECK(crsolve_set_workspace(ph, wsp, wsh) == CRSOLVE_OK, "set_workspace host");
    CHECK(crsolve_solve_host(ph, k, A, N > 1 ? B : NULL, y, x2, NULL) == CRSOLVE_OK, "solve_host");
    CHECK(memcmp(x, x2, ny * sizeof *x) == 0, "host-buffer x differs from the device path");
    printf("host-buffer path: bit-identical\n");

    /* an indefinite system: the breakdown is reported and x is NaN */
    for (int r = 0; r < m; ++r) A[((N / 2) * m + r) * m + r].re -= 3.0 * (m + 2.0);
    cudaMemcpy(dA, A, nA * sizeof *A, cudaMemcpyHostToDevice);
    CHECK(crsolve_factor(p, dA, dB, NULL) == CRSOLVE_OK, "factor indefinite");
    CHECK(crsolve_solve(p, k, dy, dx, NULL) == CRSOLVE_OK, "solve indefinite");
    CHECK(crsolve_info_get(p, &info, NULL) == CRSOLVE_OK && info.status == CRSOLVE_NOT_PD, "breakdown not reported");
    cudaMemcpy(x, dx, ny * sizeof *x, cudaMemcpyDeviceToHost);
    CHECK(isnan(x[0].re) && isnan(x[ny - 1].im), "x not NaN after a breakdown");
    printf("breakdown: level %d block %lld original block %lld\n", info.level, (long long)info.block,
           (long long)info.orig_block);

    crsolve_destroy(p);
    crsolve_destroy(ph);
    cudaFree(ws);
    cudaFree(wsp);
    cudaFree(dA);
    cudaFree(dB);
    cudaFree(dy);
    cudaFree(dx);
    free(A); free(B); free(y); free(x); free(x2);
    printf("ok\n");
    return 0;
}
