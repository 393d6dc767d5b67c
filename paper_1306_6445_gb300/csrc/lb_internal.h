// Private declarations shared by the library's translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <cmath>

#include <nvtx3/nvToolsExt.h>

#include "lb.h"

namespace lbm {

// NVTX range over the host side of an entry point (named in profiler timelines; a few
// nanoseconds when no tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

// Error bits written by kernels into the context's device flag word.
enum : int { ERR_DOMAIN = 1, ERR_TIMEOUT = 2 };

// Order of the population planes in a stored state buffer: grouped by the row each
// population is pulled from in a step (f_a(x, y) = g_a(x - e_a)): the planes of 2, 5, 6
// (pulled from row y - 1), then 0, 1, 3 (row y), then 4, 7, 8 (row y + 1). Population a of
// the state lives in plane plane_of(a); host arrays keep the natural order 0..8.
__host__ __device__ constexpr int plane_of(int a) {
    return a == 2 ? 0 : a == 5 ? 1 : a == 6 ? 2 : a == 0 ? 3 : a == 1 ? 4 : a == 3 ? 5
         : a == 4 ? 6 : a;
}

// Elements in front of column 0 of every stored row (the last two hold periodic images or
// edge copies). FP32 uses 8, so that column 0 sits 32 bytes into the row and each warp's
// 64-column store covers whole 32-byte sectors; the TMA box (columns x0 - 4 ..) then starts
// at element x0 + 4, still 16-byte aligned. FP64 rows are sector-aligned with 4 already,
// and BF16 keeps 4 because its box start must stay a multiple of 8 elements.
constexpr int ghost_of_prec(int prec) { return prec == LB_FP32 ? 8 : 4; }

// Per-lattice constants of the update, in double; kernels convert them to their type.
struct Consts {
    int eos_kind;
    // Carnahan-Starling: p = rho RT (1 + eta + eta^2 - eta^3)/(1 - eta)^3 - a rho^2, eta = b4 rho
    double a, b4, RT;
    // exponential potential psi0 exp(-rho0/rho)
    double psi0, rho0;
    // Eq. 23 branches; p_rho1 = rho1 th_v, p_rho2 = p_rho1 + (rho2 - rho1) th_m
    double th_v, th_m, th_l, rho1, rho2, p_rho1, p_rho2;
    // psi^2 = (p - rho/3) * two_over_G for the EOS-based potentials
    double two_over_G;
    double G;       // interaction strength of Eq. 7
    double kG2;     // kappa G / 2 of Eq. 19
    double sig_coef;  // 12 sigma G^2 / (tau_e - 1/2): Eq. 8 with |F|^2/psi^2 = G^2 |sum w psi e|^2
    double s_e, s_z, s_q, s_v;  // non-conserved relaxation rates (s_rho, s_j drop out, see kernels)
    int stall_row;  // test hook: the step kernel never requests this ring row (INT_MIN = off)
    double shift_rho;  // rho_s of the LB_BF16 storage shift f_a - w_a rho_s (0 otherwise)
    int stochastic;    // LB_BF16: 1 = stochastic rounding of the stored values (0 = nearest)
    unsigned step_key; // the step a launch takes (the stochastic-rounding counter)
    // nu(rho) of the open-boundary kernels: s_v_vapour where rho < rho_sw (-inf: off)
    double rho_sw, s_v_vapour;
};

// Geometry of one lattice's device population buffer.
struct Geom {
    int nx, ny;
    int pitch;          // elements per stored row (>= nx + 2 * ghost, multiple of 32)
    long long plane;    // elements per population plane = ny * pitch
    int walls;          // boundary kind (lb_bc): 0 periodic, 1 walls in y, 2 open (see lb.h)
};

// One work item of the batched step: a strip of one lattice.
struct BatchItem {
    int lat;            // lattice index
    int x0, w;          // first column (a multiple of 4) and width (<= the kernel's TX)
    int yb, n, dir;     // first row, row count, march direction (+1 / -1)
};

struct StepLaunch {
    int variant;        // compiled (strip width, ring depth) choice, see step_variant_tx
    int tx;             // lattice columns per CTA (two per thread)
    int rows;           // rows each CTA marches over
    int ctas_per_sm;    // resident CTAs per SM reported by the occupancy calculator
};

// ---- kernels (lb_kernels.cu) -------------------------------------------------------
int step_variant_count();
int step_variant_tx(int variant);
int step_variant_planes(int variant);   // population planes per TMA box (9 or 3)
int default_step_variant();
StepLaunch make_step_launch(int prec, int eos_kind, const Geom &g, int num_sms, int variant,
                            int rows_override);
cudaError_t configure_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l);
// tensor_map_in: a CUtensorMap describing the input buffer (3-D: x, y, population plane).
// Step units, one per storage type and ring kind K (lb_step_<type>.cu: K = 0, whole-row
// ring; lb_step_<type>_stage.cu: K = 1, stage ring); configure: set the kernel attributes
// only. A variant of the other kind returns cudaErrorInvalidValue (occupancy 0).
#define LB_DECLARE_STEP_UNIT(NAME, K)                                                         \
    cudaError_t step_##NAME##_k##K(const Consts &c, const Geom &g, const StepLaunch &l,      \
                                   int order, const void *tensor_map_in, void *gout, int *err, \
                                   cudaStream_t st, bool configure);                         \
    int occupancy_##NAME##_k##K(int variant, int eos_kind, int bc);
LB_DECLARE_STEP_UNIT(f32, 0)
LB_DECLARE_STEP_UNIT(f32, 1)
LB_DECLARE_STEP_UNIT(f64, 0)
LB_DECLARE_STEP_UNIT(f64, 1)
LB_DECLARE_STEP_UNIT(bf16, 0)
LB_DECLARE_STEP_UNIT(bf16, 1)
#undef LB_DECLARE_STEP_UNIT
int step_variant_kind(int variant);   // 0: whole-row ring, 1: stage ring
// batched-step units (lb_batch_kernels.cu: K = 0, lb_batch_stage.cu: K = 1)
#define LB_DECLARE_BATCH_UNIT(NAME, K)                                                        \
    cudaError_t batch_##NAME##_k##K(int variant, int eos, bool configure, int *occ, int grid, \
                                    const void *maps, const void *lats, const BatchItem *items, \
                                    int n_items, int phase, int *errs, cudaStream_t st);
LB_DECLARE_BATCH_UNIT(f32, 0)
LB_DECLARE_BATCH_UNIT(f32, 1)
LB_DECLARE_BATCH_UNIT(f64, 0)
LB_DECLARE_BATCH_UNIT(f64, 1)
#undef LB_DECLARE_BATCH_UNIT

// order 0 / 1: visit the row blocks (and the rows inside them) forward / in reverse
cudaError_t launch_step(int prec, const Consts &c, const Geom &g, const StepLaunch &l, int order,
                        const void *tensor_map_in, void *gout, int *err, cudaStream_t stream);
// packed: f in the host layout [a][y][x] (no pitch, no ghosts) instead of the padded one
cudaError_t launch_unstream(int prec, const Geom &g, const void *f, void *gbuf, bool packed,
                            cudaStream_t stream);
cudaError_t launch_stream(int prec, const Geom &g, const void *gbuf, void *f, bool packed,
                          cudaStream_t stream);
cudaError_t launch_init_feq(int prec, const Consts &c, const Geom &g, const double *rho,
                            const double *ux, const double *uy, void *f, int *err,
                            cudaStream_t stream);
// psi: nx*ny elements of the storage type
cudaError_t launch_psi_field(int prec, const Consts &c, const Geom &g, const void *gbuf,
                             void *psi, int *err, cudaStream_t stream);
cudaError_t launch_macro_fields(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                const void *psi, double *rho, double *ux, double *uy,
                                cudaStream_t stream);
// Deterministic FP64 reduction: partials must hold 4 * reduce_blocks(n) doubles.
int reduce_blocks(long long n_sites);
cudaError_t launch_macro_reduce(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                const void *psi, double *partials, double *out4,
                                cudaStream_t stream);

// Laplace sums of a droplet (8 doubles into out8, layout of k_droplet_sums); partials must
// hold 8 * reduce_blocks(n) doubles
cudaError_t launch_droplet_sums(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                double cx, double cy, double r_in, double r_out,
                                double *partials, double *out8, cudaStream_t stream);
// interface height of every column into h (nx doubles); first: nx ints of scratch
cudaError_t launch_interface_height(int prec, const Consts &c, const Geom &g, const void *gbuf,
                                    double rho_mid, int *first, double *h, cudaStream_t stream);

// Laplace-law results from the 8 sums of a droplet measurement (the layout of
// lb_batch_measure / lb_measure_droplet's out): theta, rho_in, rho_out, R (from the mass),
// p_in, p_out, mass, failed
inline void droplet_results(const double m[8], double n_sites, bool failed, double o[8]) {
    const double rho_in = m[2] > 0 ? m[1] / m[2] : NAN;
    const double rho_out = m[4] > 0 ? m[3] / m[4] : NAN;
    const double p_in = m[2] > 0 ? m[5] / m[2] : NAN;
    const double p_out = m[4] > 0 ? m[6] / m[4] : NAN;
    const double R = std::sqrt((m[0] - rho_out * n_sites) /
                               (3.14159265358979323846 * (rho_in - rho_out)));
    o[0] = (p_in - p_out) * R;
    o[1] = rho_in;
    o[2] = rho_out;
    o[3] = R;
    o[4] = p_in;
    o[5] = p_out;
    o[6] = m[0];
    o[7] = (failed || m[7] > 0 || !std::isfinite(o[0])) ? 1.0 : 0.0;
}

// ---- batched step (lb_kernels.cu) --------------------------------------------------------
// maps: 2 CUtensorMap per lattice (buffer 0, buffer 1); lats: BatchLattice<T> table
cudaError_t configure_batch(int prec, int eos_kind, int variant, int *ctas_per_sm);
cudaError_t launch_batch_step(int prec, int eos_kind, int variant, int grid, const void *maps,
                              const void *lats, const BatchItem *items, int n_items, int phase,
                              int *errs, cudaStream_t stream);
// per lattice: out[8*i ..] = mass, sum rho (r < R/2), count, sum rho (outside), count,
// sum p (inside), sum p (outside), non-finite count; FP64, fixed order
cudaError_t launch_batch_measure(int prec, int eos_kind, const void *lats, int n_lat, int phase,
                                 const double *radius, double *out, cudaStream_t stream);

// ---- read-only view of a context for entry points outside lb_api.cu (lb_noalloc.cu) ---
struct CtxView {
    const void *g;        // device buffer holding the current state
    Geom geom;
    Consts consts;
    int prec;
    cudaStream_t stream;
    lb_status sticky;
};
lb_status ctx_view(const lb_ctx *c, CtxView *v);
// record a message; with poison = true also make `s` the context's sticky status
lb_status ctx_fail(lb_ctx *c, lb_status s, const char *msg, bool poison);
// wait for the context's stream and fold the device error bits that its kernels set
// (ERR_TIMEOUT, ERR_DOMAIN) into its sticky status, exactly as every synchronising entry
// point of lb_api.cu does; allocates nothing
lb_status ctx_sync_check(lb_ctx *c);

// ---- host thermodynamics (lb_thermo.cpp) ---------------------------------------------
double p_eos_host(const lb_eos &e, double G, double rho);

}  // namespace lbm
