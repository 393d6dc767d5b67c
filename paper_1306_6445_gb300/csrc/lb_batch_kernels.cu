// Batched-lattice kernels: the persistent step over work items with the whole-row ring
// (FP32, FP64; the stage ring is in lb_batch_stage.cu) and the per-lattice Laplace
// measurement.
#include "lb_step.cuh"

namespace lbm {

namespace {

// Per-lattice Laplace sums for the batched sweep: one CTA per lattice, fixed per-thread
// order and fixed tree (deterministic). Inside: r < R/2; outside: r > R + 0.3 min(nx,ny)/2,
// around the lattice centre ((nx-1)/2, (ny-1)/2); p = rho/3 + (G/2) psi^2.
template <typename T, int EOS>
__global__ void __launch_bounds__(RED_THREADS)
k_batch_measure(const BatchLattice<T> *__restrict__ lats, int phase,
                const double *__restrict__ radius, double *__restrict__ out) {
    __shared__ double s[8][RED_THREADS];
    const BatchLattice<T> &L = lats[blockIdx.x];
    const DevConsts<T> P = L.P;
    const int nx = L.nx, ny = L.ny;
    const T *g = L.g[L.frozen ? 0 : phase];
    const double R = radius[blockIdx.x];
    const double cx = 0.5 * (nx - 1), cy = 0.5 * (ny - 1);
    const double r_in = 0.5 * R, r_out = R + 0.3 * 0.5 * min(nx, ny);
    double acc[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    const long long n = (long long)nx * ny;
    for (long long i = threadIdx.x; i < n; i += RED_THREADS) {
        const int y = (int)(i / nx), x = (int)(i % nx);
        T v[9];
#pragma unroll
        for (int a = 0; a < 9; ++a)
            v[a] = pull_global<T, false>(g, a, x, y, nx, ny, L.pitch, (long long)L.plane);
        const T rho = sum9(v);
        bool bad = false;
        const T psi = eos_psi<T, EOS>(rho, P, bad);
        const double dr = double(rho);
        const double p = dr / 3.0 + 0.5 * double(P.G) * double(psi) * double(psi);
        acc[0] += dr;
        const double r = sqrt((x - cx) * (x - cx) + (y - cy) * (y - cy));
        if (r < r_in) { acc[1] += dr; acc[2] += 1; acc[5] += p; }
        if (r > r_out) { acc[3] += dr; acc[4] += 1; acc[6] += p; }
        if (bad || !(dr == dr) || !(p == p)) acc[7] += 1;
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) s[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int wdt = RED_THREADS / 2; wdt > 0; wdt >>= 1) {
        if (threadIdx.x < wdt) {
#pragma unroll
            for (int q = 0; q < 8; ++q) s[q][threadIdx.x] += s[q][threadIdx.x + wdt];
        }
        __syncthreads();
    }
    if (threadIdx.x < 8) out[blockIdx.x * 8 + threadIdx.x] = s[threadIdx.x][0];
}

}  // namespace

cudaError_t launch_batch_measure(int prec, int eos_kind, const void *lats, int n_lat, int phase,
                                 const double *radius, double *out, cudaStream_t st) {
#define LB_BM(T, EOSK)                                                                         \
    k_batch_measure<T, EOSK><<<n_lat, RED_THREADS, 0, st>>>(                                   \
        static_cast<const BatchLattice<T> *>(lats), phase, radius, out)
    if (prec == LB_FP32) {
        if (eos_kind == LB_EOS_CS) LB_BM(float, LB_EOS_CS);
        else if (eos_kind == LB_EOS_EXP) LB_BM(float, LB_EOS_EXP);
        else LB_BM(float, LB_EOS_PIECEWISE);
    } else {
        if (eos_kind == LB_EOS_CS) LB_BM(double, LB_EOS_CS);
        else if (eos_kind == LB_EOS_EXP) LB_BM(double, LB_EOS_EXP);
        else LB_BM(double, LB_EOS_PIECEWISE);
    }
#undef LB_BM
    return cudaGetLastError();
}


LB_BATCH_UNIT(f32, float, 0)
LB_BATCH_UNIT(f64, double, 0)

}  // namespace lbm
