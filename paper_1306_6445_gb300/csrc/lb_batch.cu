// Batched lattices (lb_batch_*): many independent periodic droplet lattices of uneven size
// and parameters advanced together by one persistent kernel per time step (k_batch_step),
// replayed from a captured CUDA graph, plus per-lattice Laplace measurements on the GPU.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "lb_device.cuh"
#include "lb_internal.h"

namespace {

constexpr int kGraphSteps = 64;   // steps per captured graph (even: the phase returns)

struct BatchCommon {
    int n = 0;
    int prec = LB_FP32;
    int eos_kind = LB_EOS_CS;
    size_t elem = 4;
    cudaStream_t stream = nullptr;
    std::vector<lbm::Geom> geom;
    std::vector<lbm::Consts> consts;
    std::vector<size_t> off[2];          // byte offsets of each lattice's two buffers
    void *pool = nullptr;                // all population buffers
    void *d_maps = nullptr;              // 2 CUtensorMap per lattice
    void *d_lats = nullptr;              // BatchLattice<T> table
    lbm::BatchItem *d_items = nullptr;
    int n_items = 0;
    int *d_errs = nullptr;
    double *d_stage = nullptr;           // rho, ux, uy staging for one lattice
    size_t stage_sites = 0;
    double *d_radius = nullptr;
    double *d_meas = nullptr;
    int variant = 0, rows = 16, grid = 0, ctas_per_sm = 1, num_sms = 0;
    int phase = 0;                       // which buffer holds the active lattices' state
    std::vector<unsigned char> active;   // lattices stepped by lb_batch_step
    std::vector<long long> lat_steps;    // steps taken by each lattice
    long long steps = 0;
    cudaGraphExec_t graph[2] = {nullptr, nullptr};   // kGraphSteps steps from phase 0 / 1
    lb_status sticky = LB_OK;
    std::string msg;
};

}  // namespace

struct lb_batch : BatchCommon {};

namespace {

lb_status bfail(lb_batch *b, lb_status s, const std::string &m, bool poison = false) {
    if (b) {
        b->msg = m;
        if (poison) b->sticky = s;
    }
    return s;
}

#define LB_BCUDA(b, call)                                                            \
    do {                                                                             \
        cudaError_t e__ = (call);                                                    \
        if (e__ != cudaSuccess)                                                      \
            return bfail(b, LB_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e__)); \
    } while (0)

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn batch_encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
    }
    return fn;
}

void *buf(lb_batch *b, int i, int which) {
    return static_cast<char *>(b->pool) + b->off[which][i];
}

// Work items for a strip width `tx` and `rows` rows per item: each lattice is cut into
// ceil(nx / tx) strips (lb_strip_widths) and row blocks of `rows` rows marching
// alternately up and down; items are ordered lattice by lattice so that the neighbours of
// a row block run at the same time. Every strip starts on a multiple of 4 columns (the
// TMA start coordinate must be 16-byte aligned); an item that would not is refused.
bool make_items(const lb_batch *b, int tx, int rows, std::vector<lbm::BatchItem> &items) {
    items.clear();
    std::vector<int> widths(4096);
    for (int i = 0; i < b->n; ++i) {
        if (!b->active[i]) continue;     // an inactive lattice has no work items
        const int nx = b->geom[i].nx, ny = b->geom[i].ny;
        const int ns = lb_strip_widths(nx, tx, widths.data(), (int)widths.size());
        if (ns <= 0) return false;
        const int nb = (ny + rows - 1) / rows;
        for (int rb = 0; rb < nb; ++rb) {
            int x0 = 0;
            for (int k = 0; k < ns; ++k) {
                lbm::BatchItem it;
                it.lat = i;
                it.x0 = x0;
                it.w = widths[k];
                it.yb = rb * rows;
                it.n = std::min(rows, ny - it.yb);
                it.dir = (rb & 1) ? -1 : 1;
                if ((it.x0 & 3) != 0 || it.w < 1 || it.w > tx || it.x0 + it.w > nx || it.n < 1)
                    return false;
                items.push_back(it);
                x0 += widths[k];
            }
        }
    }
    return true;
}

void drop_graphs(lb_batch *b) {
    for (auto &g : b->graph) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
}

lb_status apply_batch_launch(lb_batch *b, int variant, int rows) {
    if (variant < 0 || variant >= lbm::step_variant_count())
        return bfail(b, LB_EINVAL, "unknown launch variant");
    if (rows <= 0) rows = 16;
    const int tx = lbm::step_variant_tx(variant);
    int occ = 0;
    LB_BCUDA(b, lbm::configure_batch(b->prec, b->eos_kind, variant, &occ));
    std::vector<lbm::BatchItem> items;
    if (!make_items(b, tx, rows, items)) return bfail(b, LB_EINVAL, "bad strip decomposition");
    if (b->d_items) cudaFree(b->d_items);
    b->d_items = nullptr;
    LB_BCUDA(b, cudaMalloc(&b->d_items, items.size() * sizeof(lbm::BatchItem)));
    LB_BCUDA(b, cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(lbm::BatchItem),
                           cudaMemcpyHostToDevice));
    b->n_items = (int)items.size();
    b->variant = variant;
    b->rows = rows;
    b->ctas_per_sm = std::max(occ, 1);
    b->grid = std::min(b->n_items, b->num_sms * b->ctas_per_sm);
    // tensor maps: the box width follows the strip width of the variant
    EncodeTiledFn enc = batch_encode_fn();
    if (!enc) return bfail(b, LB_ECUDA, "cuTensorMapEncodeTiled unavailable");
    std::vector<CUtensorMap> maps(2 * (size_t)b->n);
    const CUtensorMapDataType dt =
        b->prec == LB_FP32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64;
    for (int i = 0; i < b->n; ++i) {
        const lbm::Geom &g = b->geom[i];
        const cuuint64_t dims[3] = {(cuuint64_t)g.pitch, (cuuint64_t)g.ny, 9};
        const cuuint64_t strides[2] = {(cuuint64_t)g.pitch * b->elem, (cuuint64_t)g.plane * b->elem};
        const cuuint32_t box[3] = {(cuuint32_t)(tx + lbm::ghost_of_prec(b->prec) + 4), 1,
                                   (cuuint32_t)lbm::step_variant_planes(variant)};
        const cuuint32_t estr[3] = {1, 1, 1};
        for (int w = 0; w < 2; ++w) {
            CUresult r = enc(&maps[2 * i + w], dt, 3, buf(b, i, w), dims, strides, box, estr,
                             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS) return bfail(b, LB_ECUDA, "cuTensorMapEncodeTiled failed");
        }
    }
    LB_BCUDA(b, cudaMemcpy(b->d_maps, maps.data(), maps.size() * sizeof(CUtensorMap),
                           cudaMemcpyHostToDevice));
    drop_graphs(b);
    return LB_OK;
}

// the buffer holding lattice i's state: an inactive lattice was set inactive at an even
// step count, so its state stays in buffer 0
int cur(const lb_batch *b, int i) { return b->active[i] ? b->phase : 0; }

template <typename T>
lb_status upload_lattices(lb_batch *b) {
    std::vector<lbm::BatchLattice<T>> t(b->n);
    for (int i = 0; i < b->n; ++i) {
        t[i].g[0] = static_cast<T *>(buf(b, i, 0));
        t[i].g[1] = static_cast<T *>(buf(b, i, 1));
        t[i].P = lbm::to_dev<T>(b->consts[i]);
        t[i].nx = b->geom[i].nx;
        t[i].ny = b->geom[i].ny;
        t[i].pitch = b->geom[i].pitch;
        t[i].plane = (unsigned)b->geom[i].plane;
        t[i].frozen = b->active[i] ? 0 : 1;
    }
    if (!b->d_lats) LB_BCUDA(b, cudaMalloc(&b->d_lats, t.size() * sizeof(t[0])));
    LB_BCUDA(b, cudaMemcpy(b->d_lats, t.data(), t.size() * sizeof(t[0]), cudaMemcpyHostToDevice));
    return LB_OK;
}

void count_steps(lb_batch *b, int n) {
    b->steps += n;
    for (int i = 0; i < b->n; ++i)
        if (b->active[i]) b->lat_steps[i] += n;
}

lb_status launch_steps(lb_batch *b, int n) {
    for (int i = 0; i < n; ++i) {
        if (b->n_items > 0)
            LB_BCUDA(b, lbm::launch_batch_step(b->prec, b->eos_kind, b->variant, b->grid,
                                               b->d_maps, b->d_lats, b->d_items, b->n_items,
                                               b->phase, b->d_errs, b->stream));
        b->phase ^= 1;
        count_steps(b, 1);
    }
    return LB_OK;
}

lb_status ensure_graph(lb_batch *b, int phase) {
    if (b->graph[phase]) return LB_OK;
    cudaStream_t cap = nullptr;
    LB_BCUDA(b, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i)
            e = lbm::launch_batch_step(b->prec, b->eos_kind, b->variant, b->grid, b->d_maps,
                                       b->d_lats, b->d_items, b->n_items, phase ^ (i & 1),
                                       b->d_errs, cap);
        cudaError_t e2 = cudaStreamEndCapture(cap, &g);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->graph[phase], g, 0);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess)
        return bfail(b, LB_ECUDA, std::string("graph capture: ") + cudaGetErrorString(e));
    return LB_OK;
}

lb_status batch_sync(lb_batch *b) {
    LB_BCUDA(b, cudaStreamSynchronize(b->stream));
    std::vector<int> errs(b->n);
    LB_BCUDA(b, cudaMemcpy(errs.data(), b->d_errs, b->n * sizeof(int), cudaMemcpyDeviceToHost));
    int any = 0;
    for (int v : errs) any |= v;
    if (any & lbm::ERR_TIMEOUT)
        return bfail(b, LB_ETIMEOUT, "a bounded device-side wait gave up", true);
    return LB_OK;   // per-lattice domain errors are reported by lb_batch_errors
}

}  // namespace

extern "C" {

int lb_strip_widths(int nx, int tx, int *widths, int max_strips) {
    if (nx < 1 || tx < 4 || (tx & 3) || !widths) return -1;
    const int ns = (nx + tx - 1) / tx;
    if (ns > max_strips) return -1;
    // m groups of 4 columns (the last one possibly partial) spread as evenly as possible;
    // every strip but the last is a whole number of groups, so all starts are multiples of 4
    const int m = (nx + 3) / 4;
    int used = 0;
    for (int k = 0; k < ns; ++k) {
        const int g = m / ns + (k < m % ns ? 1 : 0);
        widths[k] = 4 * g;
        used += widths[k];
    }
    widths[ns - 1] -= used - nx;   // drop the unused part of the last group
    return ns;
}

lb_status lb_batch_create(lb_batch **out, int n, const lb_lattice_desc *descs, int prec,
                          void *stream) {
    if (!out || n <= 0 || !descs) return LB_EINVAL;
    *out = nullptr;
    if (prec != LB_FP32 && prec != LB_FP64) return LB_EINVAL;
    lb_batch *b = new (std::nothrow) lb_batch();
    if (!b) return LB_ENOMEM;
    b->n = n;
    b->prec = prec;
    b->elem = prec == LB_FP32 ? 4 : 8;
    b->stream = static_cast<cudaStream_t>(stream);
    b->eos_kind = descs[0].eos.kind;
    size_t total = 0;
    for (int i = 0; i < n; ++i) {
        const lb_lattice_desc &d = descs[i];
        if (d.eos.kind != b->eos_kind || d.nx < 3 || d.ny < 3 ||
            9LL * (long long)lb_pitch(d.nx, prec) * d.ny >= (1LL << 32)) {
            delete b;
            return LB_EINVAL;
        }
        if (!(d.kappa >= 0 && d.kappa < 1) || !(d.sigma_force >= 0) ||
            (d.sigma_force != 0 && d.rates.s_zeta != d.rates.s_e)) {
            delete b;
            return LB_EINVAL;
        }
        const double r[6] = {d.rates.s_rho, d.rates.s_e, d.rates.s_zeta, d.rates.s_j,
                             d.rates.s_q, d.rates.s_v};
        for (double s : r)
            if (!(s > 0 && s < 2)) {
                delete b;
                return LB_EINVAL;
            }
        if (d.eos.kind != LB_EOS_EXP && d.G == 0.0) {
            delete b;
            return LB_EINVAL;
        }
        lbm::Geom g;
        g.nx = d.nx;
        g.ny = d.ny;
        g.pitch = (int)lb_pitch(d.nx, prec);
        g.plane = (long long)d.ny * g.pitch;
        g.walls = 0;
        b->geom.push_back(g);
        lbm::Consts c{};
        c.eos_kind = d.eos.kind;
        c.a = d.eos.a;
        c.b4 = d.eos.b / 4.0;
        c.RT = d.eos.R * d.eos.T;
        c.psi0 = d.eos.psi0;
        c.rho0 = d.eos.rho0;
        c.th_v = d.eos.theta_v;
        c.th_m = d.eos.theta_m;
        c.th_l = d.eos.theta_l;
        c.rho1 = d.eos.rho1;
        c.rho2 = d.eos.rho2;
        c.p_rho1 = d.eos.rho1 * d.eos.theta_v;
        c.p_rho2 = c.p_rho1 + (d.eos.rho2 - d.eos.rho1) * d.eos.theta_m;
        c.two_over_G = d.G != 0 ? 2.0 / d.G : 0.0;
        c.G = d.G;
        c.kG2 = d.kappa * d.G / 2.0;
        c.sig_coef = 12.0 * d.sigma_force * d.G * d.G / (1.0 / d.rates.s_e - 0.5);
        c.s_e = d.rates.s_e;
        c.s_z = d.rates.s_zeta;
        c.s_q = d.rates.s_q;
        c.s_v = d.rates.s_v;
        c.stall_row = INT_MIN;
        c.rho_sw = -HUGE_VAL;       // nu(rho) off
        c.s_v_vapour = c.s_v;
        b->consts.push_back(c);
        const size_t bytes = (lb_buffer_bytes(d.nx, d.ny, prec) + 255) / 256 * 256;
        for (int w = 0; w < 2; ++w) {
            b->off[w].push_back(total);
            total += bytes;
        }
        b->stage_sites = std::max(b->stage_sites, (size_t)d.nx * d.ny);
    }
    int dev = 0;
    lb_status s = LB_OK;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaMalloc(&b->pool, total) != cudaSuccess ||
        cudaMalloc(&b->d_maps, 2 * (size_t)n * sizeof(CUtensorMap)) != cudaSuccess ||
        cudaMalloc(&b->d_errs, n * sizeof(int)) != cudaSuccess ||
        cudaMalloc(&b->d_stage, 3 * b->stage_sites * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_radius, n * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&b->d_meas, 8 * (size_t)n * sizeof(double)) != cudaSuccess ||
        cudaMemset(b->pool, 0, total) != cudaSuccess ||
        cudaMemset(b->d_errs, 0, n * sizeof(int)) != cudaSuccess) {
        lb_batch_free(b);
        return LB_ENOMEM;
    }
    b->active.assign(n, 1);
    b->lat_steps.assign(n, 0);
    s = prec == LB_FP32 ? upload_lattices<float>(b) : upload_lattices<double>(b);
    if (s == LB_OK) s = apply_batch_launch(b, lbm::default_step_variant(), 16);
    if (s != LB_OK) {
        std::fprintf(stderr, "lb_batch_create: %s\n", b->msg.c_str());
        lb_batch_free(b);
        return s;
    }
    *out = b;
    return LB_OK;
}

lb_status lb_batch_set_launch(lb_batch *b, int variant, int rows) {
    if (!b) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    LB_BCUDA(b, cudaStreamSynchronize(b->stream));
    return apply_batch_launch(b, variant, rows);
}

lb_status lb_batch_get_launch(const lb_batch *b, int *variant, int *rows, int *grid,
                              int *items) {
    if (!b) return LB_EINVAL;
    if (variant) *variant = b->variant;
    if (rows) *rows = b->rows;
    if (grid) *grid = b->grid;
    if (items) *items = b->n_items;
    return LB_OK;
}

lb_status lb_batch_autotune(lb_batch *b, int trial_steps, int *variant, int *rows) {
    if (!b) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    if (trial_steps < 2) trial_steps = 2;
    // the trial launches take real steps of the current states: the pool, the error flags,
    // the phase and the step count are saved first and restored afterwards
    const size_t total = b->off[1].back() +
                         (lb_buffer_bytes(b->geom.back().nx, b->geom.back().ny, b->prec) + 255) / 256 * 256;
    void *saved = nullptr;
    int *saved_errs = nullptr;
    if (cudaMalloc(&saved, total) != cudaSuccess) {
        cudaGetLastError();
        return bfail(b, LB_ENOMEM, "lb_batch_autotune: no device memory for the state copy");
    }
    if (cudaMalloc(&saved_errs, b->n * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        cudaFree(saved);
        return bfail(b, LB_ENOMEM, "lb_batch_autotune: no device memory for the state copy");
    }
    const int phase0 = b->phase;
    const long long steps0 = b->steps;
    const std::vector<long long> lat_steps0 = b->lat_steps;
    const int v0 = b->variant, r0 = b->rows;
    cudaError_t e = cudaMemcpyAsync(saved, b->pool, total, cudaMemcpyDeviceToDevice, b->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(saved_errs, b->d_errs, b->n * sizeof(int), cudaMemcpyDeviceToDevice,
                            b->stream);
    const int cand_rows[] = {8, 12, 16, 24, 32};
    float best = 1e30f;
    int bv = v0, br = r0;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    for (int v = 0; v < lbm::step_variant_count() && e == cudaSuccess; ++v) {
        for (int r : cand_rows) {
            if (apply_batch_launch(b, v, r) != LB_OK) continue;
            if (launch_steps(b, 1) != LB_OK) continue;                 // warm-up
            cudaEventRecord(e0, b->stream);
            if (launch_steps(b, trial_steps) != LB_OK) continue;
            cudaEventRecord(e1, b->stream);
            e = cudaEventSynchronize(e1);
            float ms = 0;
            if (e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
            if (ms > 0 && ms < best) {
                best = ms;
                bv = v;
                br = r;
            }
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    // put the states back (whatever the trials did)
    cudaError_t e2 = cudaMemcpyAsync(b->pool, saved, total, cudaMemcpyDeviceToDevice, b->stream);
    if (e2 == cudaSuccess)
        e2 = cudaMemcpyAsync(b->d_errs, saved_errs, b->n * sizeof(int), cudaMemcpyDeviceToDevice,
                             b->stream);
    if (e2 == cudaSuccess) e2 = cudaStreamSynchronize(b->stream);
    cudaFree(saved);
    cudaFree(saved_errs);
    b->phase = phase0;
    b->steps = steps0;
    b->lat_steps = lat_steps0;
    if (e != cudaSuccess) return bfail(b, LB_ECUDA, cudaGetErrorString(e));
    if (e2 != cudaSuccess) return bfail(b, LB_ECUDA, cudaGetErrorString(e2));
    lb_status s = apply_batch_launch(b, bv, br);
    if (s != LB_OK) return s;
    if (variant) *variant = bv;
    if (rows) *rows = br;
    return LB_OK;
}

lb_status lb_batch_set_rho_u(lb_batch *b, int i, const double *rho, const double *ux,
                             const double *uy) {
    if (!b || i < 0 || i >= b->n || !rho || !ux || !uy) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    const lbm::Geom &g = b->geom[i];
    const size_t n = (size_t)g.nx * g.ny;
    LB_BCUDA(b, cudaMemcpyAsync(b->d_stage, rho, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    LB_BCUDA(b, cudaMemcpyAsync(b->d_stage + n, ux, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    LB_BCUDA(b, cudaMemcpyAsync(b->d_stage + 2 * n, uy, n * sizeof(double), cudaMemcpyHostToDevice, b->stream));
    // the per-lattice error word doubles as the init kernel's domain flag
    LB_BCUDA(b, lbm::launch_init_feq(b->prec, b->consts[i], g, b->d_stage, b->d_stage + n,
                                     b->d_stage + 2 * n, buf(b, i, cur(b, i) ^ 1), b->d_errs + i,
                                     b->stream));
    LB_BCUDA(b, lbm::launch_unstream(b->prec, g, buf(b, i, cur(b, i) ^ 1), buf(b, i, cur(b, i)),
                                     false, b->stream));
    LB_BCUDA(b, cudaStreamSynchronize(b->stream));
    int e = 0;
    LB_BCUDA(b, cudaMemcpy(&e, b->d_errs + i, sizeof(int), cudaMemcpyDeviceToHost));
    if (e & lbm::ERR_DOMAIN) return bfail(b, LB_EDOMAIN, "lattice density outside the EOS branch");
    return LB_OK;
}

lb_status lb_batch_step(lb_batch *b, int n) {
    const lbm::NvtxRange nvtx_range("lb_batch_step");
    if (!b || n < 0) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    while (n >= kGraphSteps) {
        if (b->n_items > 0) {
            lb_status s = ensure_graph(b, b->phase);
            if (s != LB_OK) return s;
            LB_BCUDA(b, cudaGraphLaunch(b->graph[b->phase], b->stream));
        }
        count_steps(b, kGraphSteps);   // even: the phase is unchanged
        n -= kGraphSteps;
    }
    return launch_steps(b, n);
}

lb_status lb_batch_sync(lb_batch *b) {
    if (!b) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    return batch_sync(b);
}

lb_status lb_batch_errors(lb_batch *b, int *flags) {
    if (!b || !flags) return LB_EINVAL;
    lb_status s = batch_sync(b);
    if (s != LB_OK && s != LB_ETIMEOUT) return s;
    LB_BCUDA(b, cudaMemcpy(flags, b->d_errs, b->n * sizeof(int), cudaMemcpyDeviceToHost));
    return s;
}

lb_status lb_batch_get_rho(lb_batch *b, int i, double *rho) {
    if (!b || i < 0 || i >= b->n || !rho) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    const lbm::Geom &g = b->geom[i];
    const size_t n = (size_t)g.nx * g.ny;
    LB_BCUDA(b, lbm::launch_macro_fields(b->prec, b->consts[i], g, buf(b, i, cur(b, i)), nullptr,
                                         b->d_stage, nullptr, nullptr, b->stream));
    LB_BCUDA(b, cudaMemcpyAsync(rho, b->d_stage, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
    return batch_sync(b);
}

lb_status lb_batch_get_populations(lb_batch *b, int i, void *dst, size_t bytes) {
    if (!b || i < 0 || i >= b->n || !dst) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    const lbm::Geom &g = b->geom[i];
    const size_t row = (size_t)g.nx * b->elem;
    if (bytes != 9 * (size_t)g.ny * row) return bfail(b, LB_EINVAL, "size mismatch");
    // the spare buffer of lattice i receives the pulled populations in the host layout
    // (free between steps), then one contiguous copy
    void *spare = buf(b, i, cur(b, i) ^ 1);
    LB_BCUDA(b, lbm::launch_stream(b->prec, g, buf(b, i, cur(b, i)), spare, true, b->stream));
    LB_BCUDA(b, cudaMemcpyAsync(dst, spare, bytes, cudaMemcpyDeviceToHost, b->stream));
    return batch_sync(b);
}

lb_status lb_batch_measure(lb_batch *b, const double *radius, double *out) {
    const lbm::NvtxRange nvtx_range("lb_batch_measure");
    if (!b || !radius || !out) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    LB_BCUDA(b, cudaMemcpyAsync(b->d_radius, radius, b->n * sizeof(double), cudaMemcpyHostToDevice,
                                b->stream));
    LB_BCUDA(b, lbm::launch_batch_measure(b->prec, b->eos_kind, b->d_lats, b->n, b->phase,
                                          b->d_radius, b->d_meas, b->stream));
    std::vector<double> raw(8 * (size_t)b->n);
    LB_BCUDA(b, cudaMemcpyAsync(raw.data(), b->d_meas, raw.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, b->stream));
    lb_status s = batch_sync(b);
    if (s != LB_OK) return s;
    std::vector<int> errs(b->n);
    LB_BCUDA(b, cudaMemcpy(errs.data(), b->d_errs, b->n * sizeof(int), cudaMemcpyDeviceToHost));
    for (int i = 0; i < b->n; ++i)
        lbm::droplet_results(&raw[8 * (size_t)i], (double)b->geom[i].nx * b->geom[i].ny,
                             errs[i] != 0, out + 8 * (size_t)i);
    return LB_OK;
}

lb_status lb_batch_set_active(lb_batch *b, const unsigned char *active) {
    if (!b || !active) return LB_EINVAL;
    if (b->sticky != LB_OK) return b->sticky;
    if (b->steps & 1)
        return bfail(b, LB_EINVAL, "lb_batch_set_active: call at an even step count");
    LB_BCUDA(b, cudaStreamSynchronize(b->stream));   // no queued step reads the old items
    for (int i = 0; i < b->n; ++i) b->active[i] = active[i] ? 1 : 0;
    lb_status s = b->prec == LB_FP32 ? upload_lattices<float>(b) : upload_lattices<double>(b);
    if (s != LB_OK) return s;
    return apply_batch_launch(b, b->variant, b->rows);
}

long long lb_batch_lattice_steps(const lb_batch *b, int i) {
    return (b && i >= 0 && i < b->n) ? b->lat_steps[i] : -1;
}

long long lb_batch_steps_done(const lb_batch *b) { return b ? b->steps : 0; }

int lb_batch_size(const lb_batch *b) { return b ? b->n : 0; }

const char *lb_batch_last_error(const lb_batch *b) { return b ? b->msg.c_str() : "no batch"; }

void lb_batch_free(lb_batch *b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    else cudaDeviceSynchronize();
    drop_graphs(b);
    cudaFree(b->pool);
    cudaFree(b->d_maps);
    cudaFree(b->d_lats);
    cudaFree(b->d_items);
    cudaFree(b->d_errs);
    cudaFree(b->d_stage);
    cudaFree(b->d_radius);
    cudaFree(b->d_meas);
    delete b;
}

}  // extern "C"
