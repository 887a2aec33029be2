// C-ABI entry points: argument validation, status codes, error strings and
// dispatch to the kernels. No exception crosses this boundary.
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "common.cuh"

namespace geraf {

// implemented in fields_blend.cu, phasor.cu, mlp.cu
geraf_status sample_impl(const geraf_grid*, int32_t, uint64_t, uint64_t, float*, float*, cudaStream_t);
geraf_status analytic_fields_impl(const float*, int, const float*, int64_t, float*, float*, float*, cudaStream_t);
geraf_status blend_impl(const float*, const float*, const float*, int32_t, int32_t, const float*, const float*,
                        int32_t, float, float, float*, float*, float*, float*, float*, cudaStream_t);
geraf_status blend_backward_impl(const float*, const float*, const float*, const float*, const float*, int32_t,
                                 int32_t, float, float, const float*, const float*, float*, float*, float*, void*,
                                 size_t*, cudaStream_t);
geraf_status render_impl(const float*, const float*, const float*, const float*, int64_t, const float*,
                         const float*, int32_t, const geraf_band*, int32_t, void*, size_t*, float*, cudaStream_t);
geraf_status render_backward_impl(const float*, const float*, const float*, const float*, int64_t, const float*,
                                  const float*, int32_t, const geraf_band*, int32_t, const float*, void*, size_t*,
                                  float*, float*, float*, cudaStream_t);
geraf_status render_noalloc_impl(const float*, const float*, const float*, const float*, int64_t, const float*,
                                 const float*, int32_t, const geraf_band*, int32_t, float*, cudaStream_t);
geraf_status filter_impl(const float*, const float*, int32_t, const geraf_band*, const float*, int64_t,
                         const float*, const float*, void*, size_t*, float*, float*, double*, float*, cudaStream_t);
geraf_status filter_backward_impl(const float*, int32_t, const geraf_band*, const float*, int64_t, const float*,
                                  const float*, void*, size_t*, float*, cudaStream_t);
geraf_status masked_loss_impl(const float*, const float*, float*, int64_t, float, float, void*, size_t*, double*,
                              float*, float*, cudaStream_t);
geraf_status chebyshev_order_impl(const float*, int64_t, const float*, int32_t, const geraf_band*, void*, size_t*,
                                  int32_t*, cudaStream_t);
geraf_status chebyshev_work_impl(const float*, int64_t, const float*, int32_t, const geraf_band*, int32_t, void*,
                                 size_t*, int32_t*, double*, cudaStream_t);
geraf_status mlp_saved_bytes(const geraf_field_desc*, int64_t, size_t*);
geraf_status proposal_saved_bytes(const geraf_proposal*, size_t*);
geraf_status proposal_density_impl(const geraf_proposal*, float*, float*, void*, size_t, cudaStream_t);
geraf_status sample_cells_impl(const geraf_grid*, const geraf_proposal*, const float*, int32_t, int32_t, int32_t,
                               uint64_t, uint64_t, float*, float*, int32_t*, float*, void*, size_t*, cudaStream_t);
geraf_status sample_proposal_impl(const geraf_grid*, const geraf_proposal*, const float*, uint64_t, uint64_t, float*,
                                  float*, int32_t*, cudaStream_t);
geraf_status sample_backward_impl(const geraf_proposal*, const geraf_grid*, int32_t, const float*, const float*,
                                  const int32_t*, const float*, const void*, float*, float*, double*, void*, size_t*,
                                  cudaStream_t);
geraf_status mlp_forward_impl(const geraf_field_desc*, const float*, int64_t, float*, float*, float*, void*, size_t,
                              cudaStream_t);
geraf_status mlp_backward_impl(const geraf_field_desc*, const float*, int64_t, const void*, const float*,
                               const float*, const float*, float*, void*, size_t*, cudaStream_t);

static thread_local char g_err[512] = "";

void set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

geraf_status fail(geraf_status st, const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

geraf_status cuda_status(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return GERAF_OK;
    return fail(GERAF_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

__device__ int g_device_error_word;

static std::mutex g_dev_mu;
static int* g_err_ptr[64];
static int g_sm_count[64];

static int current_device() {
    int d = 0;
    cudaGetDevice(&d);
    return d < 64 ? d : 63;
}

int* device_error_word() {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_err_ptr[d]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_device_error_word) == cudaSuccess) g_err_ptr[d] = static_cast<int*>(p);
    }
    return g_err_ptr[d];
}

// (kernel, device, bytes) opted in to large dynamic shared memory so far
struct SmemAttr {
    const void* func;
    int dev;
    int bytes;
};
static std::mutex g_attr_mu;
static std::vector<SmemAttr> g_attr_done;

geraf_status ensure_smem_attr(const void* func, int bytes, const char* what) {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_attr_mu);
    for (const SmemAttr& a : g_attr_done)
        if (a.func == func && a.dev == d && a.bytes >= bytes) return GERAF_OK;
    const cudaError_t e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e != cudaSuccess) return cuda_status(e, what);
    g_attr_done.push_back(SmemAttr{func, d, bytes});
    return GERAF_OK;
}

int device_sm_count() {
    const int d = current_device();
    std::lock_guard<std::mutex> lk(g_dev_mu);
    if (!g_sm_count[d]) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, d) != cudaSuccess || n <= 0) n = 148;
        g_sm_count[d] = n;
    }
    return g_sm_count[d];
}

bool make_band_k(const geraf_band* band, BandK* out) {
    if (!band || band->n_f < 1 || !(band->f0 > 0.0) || !(band->df >= 0.0)) {
        set_error("band: need n_f >= 1, f0 > 0, df >= 0");
        return false;
    }
    if (band->method < GERAF_PHASOR_AUTO || band->method > GERAF_PHASOR_CHEBYSHEV) {
        set_error("band: unknown method %d", band->method);
        return false;
    }
    const int g = (band->n_f + kBinsPerBlock - 1) / kBinsPerBlock;
    if (g > 32) {
        set_error("band: n_f = %d above the supported 1024", band->n_f);
        return false;
    }
    memset(out, 0, sizeof(*out));
    out->g = g;
    for (int b = 0; b < g; ++b) {
        const double K = 2.0 * (band->f0 + (double)(kBinsPerBlock * b) * band->df) / kC;
        const float hi = (float)K;
        out->k[2 * b] = hi;
        out->k[2 * b + 1] = (float)(K - (double)hi);
    }
    out->kd = (float)(2.0 * band->df / kC);
    return true;
}

}  // namespace geraf

using namespace geraf;

#define REQUIRE(cond, ...)                                      \
    do {                                                        \
        if (!(cond)) return fail(GERAF_ERR_INVALID_ARG, __VA_ARGS__); \
    } while (0)

static inline cudaStream_t S(void* s) { return static_cast<cudaStream_t>(s); }

static geraf_status check_ws(void* ws, size_t* ws_bytes) {
    if (!ws_bytes) return fail(GERAF_ERR_INVALID_ARG, "ws_bytes must not be NULL");
    if (ws && (reinterpret_cast<uintptr_t>(ws) & 255u))
        return fail(GERAF_ERR_ALIGNMENT, "workspace must be 256-byte aligned");
    return GERAF_OK;
}

extern "C" {

const char* geraf_last_error_string(void) { return g_err; }

int32_t geraf_version(void) { return 1; }

geraf_status geraf_poll_device_error(void* stream) {
    cudaError_t e = cudaStreamSynchronize(S(stream));
    if (e != cudaSuccess) return cuda_status(e, "poll_device_error");
    int* p = device_error_word();
    if (!p) return fail(GERAF_ERR_CUDA, "device error word unavailable");
    int v = 0;
    e = cudaMemcpy(&v, p, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_status(e, "poll_device_error");
    if (v) {
        int z = 0;
        cudaMemcpy(p, &z, sizeof(int), cudaMemcpyHostToDevice);
        return fail(GERAF_ERR_TIMEOUT, "a kernel gave up a bounded wait (device error word %d)", v);
    }
    return GERAF_OK;
}

namespace {
// one CTA: an mbarrier expecting one arrival that never comes; the bounded
// wait runs out, the timeout goes to the device error word
__global__ void bounded_wait_kernel(uint64_t limit_ns, int* err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    geraf::mbar_init(&bar, 1);
    geraf::fence_barrier_init();
    if (!geraf::mbar_wait(&bar, 0, limit_ns)) atomicOr(err, 1);
}
}  // namespace

geraf_status geraf_check_bounded_wait(uint64_t limit_ns, void* stream) {
    REQUIRE(limit_ns >= 1000ull && limit_ns <= 1000000000ull, "check_bounded_wait: limit_ns must be in [1e3, 1e9]");
    int* err = device_error_word();
    if (!err) return fail(GERAF_ERR_CUDA, "device error word unavailable");
    bounded_wait_kernel<<<1, 32, 0, S(stream)>>>(limit_ns, err);
    return cuda_status(cudaGetLastError(), "check_bounded_wait");
}

geraf_status geraf_sample(const geraf_grid* grid, int32_t mode, uint64_t seed, uint64_t step, float* xyz,
                          float* xyz_apr, void* stream) {
    REQUIRE(grid && xyz, "sample: grid and xyz must not be NULL");
    REQUIRE(mode == GERAF_SAMPLE_UNIFORM || mode == GERAF_SAMPLE_STRATIFIED, "sample: unknown mode %d", mode);
    for (int d = 0; d < 3; ++d) {
        REQUIRE(grid->n[d] > 0, "sample: n[%d] = %d must be positive", d, grid->n[d]);
        REQUIRE(grid->pitch[d] > 0.0f, "sample: pitch[%d] must be positive", d);
    }
    const int64_t n = (int64_t)grid->n[0] * grid->n[1] * grid->n[2];
    REQUIRE(n < (1ll << 40), "sample: %lld points exceed the 2^40 index space", (long long)n);
    REQUIRE(step < (1ull << 22), "sample: step must be below 2^22");
    return sample_impl(grid, mode, seed, step, xyz, xyz_apr, S(stream));
}

geraf_status geraf_fields_saved_bytes(const geraf_field_desc* desc, int64_t n, size_t* bytes) {
    REQUIRE(desc && bytes && n >= 0, "fields_saved_bytes: bad arguments");
    if (desc->kind == GERAF_FIELD_ANALYTIC) {
        *bytes = 0;
        return GERAF_OK;
    }
    return mlp_saved_bytes(desc, n, bytes);
}

geraf_status geraf_fields(const geraf_field_desc* desc, const float* xyz, int64_t n, float* sdf, float* grad,
                          float* refl, void* saved, size_t saved_bytes, void* stream) {
    REQUIRE(desc && xyz && sdf, "fields: desc, xyz and sdf must not be NULL");
    REQUIRE(n >= 0, "fields: n must be >= 0");
    if (n == 0) return GERAF_OK;
    if (desc->kind == GERAF_FIELD_ANALYTIC) {
        REQUIRE(desc->prims && desc->n_prims > 0 && desc->n_prims <= 1024, "fields: need 1..1024 primitives");
        return analytic_fields_impl(desc->prims, desc->n_prims, xyz, n, sdf, grad, refl, S(stream));
    }
    REQUIRE(desc->kind == GERAF_FIELD_MLP, "fields: unknown kind %d", desc->kind);
    REQUIRE(desc->params, "fields: params must not be NULL");
    return mlp_forward_impl(desc, xyz, n, sdf, grad, refl, saved, saved_bytes, S(stream));
}

geraf_status geraf_fields_backward(const geraf_field_desc* desc, const float* xyz, int64_t n, const void* saved,
                                   const float* d_sdf, const float* d_grad, const float* d_refl, float* d_params,
                                   void* ws, size_t* ws_bytes, void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(desc && desc->kind == GERAF_FIELD_MLP, "fields_backward: needs an MLP field");
    REQUIRE(n >= 1, "fields_backward: n must be >= 1");
    if (ws) REQUIRE(xyz && saved && d_params && desc->params, "fields_backward: null input or output");
    return mlp_backward_impl(desc, xyz, n, saved, d_sdf, d_grad, d_refl, d_params, ws, ws_bytes, S(stream));
}

geraf_status geraf_blend(const float* sdf, const float* refl, int32_t n_ray, int32_t n_z, const float* sdf_apr,
                         const float* sdf_ant, int32_t n_ant, float s, float a_tx, float* alpha, float* T, float* w,
                         float* t_eff, float* c_ant, const float* keep, void* stream) {
    REQUIRE(n_ray >= 1 && n_z >= 1 && n_ant >= 0, "blend: bad sizes");
    REQUIRE(sdf && refl && sdf_apr && alpha && T && w && t_eff, "blend: null input or output");
    REQUIRE(n_ant == 0 || (sdf_ant && c_ant), "blend: null antenna arrays");
    REQUIRE(s > 0.0f, "blend: sharpness s must be positive");
    return blend_impl(sdf, refl, keep, n_ray, n_z, sdf_apr, sdf_ant, n_ant, s, a_tx, alpha, T, w, t_eff, c_ant,
                      S(stream));
}

geraf_status geraf_blend_backward(const float* sdf, const float* refl, const float* alpha, const float* T,
                                  int32_t n_ray, int32_t n_z, float s, float a_tx, const float* d_w,
                                  const float* d_teff, float* d_sdf, float* d_refl, float* d_scalars,
                                  const float* keep, void* ws, size_t* ws_bytes, void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(n_ray >= 1 && n_z >= 1, "blend_backward: bad sizes");
    if (ws)
        REQUIRE(sdf && refl && alpha && T && d_sdf && d_refl && d_scalars, "blend_backward: null input or output");
    return blend_backward_impl(sdf, refl, keep, alpha, T, n_ray, n_z, s, a_tx, d_w, d_teff, d_sdf, d_refl, d_scalars,
                               ws, ws_bytes, S(stream));
}

geraf_status geraf_render(const float* xyz, const float* grad, const float* w, const float* t_eff, int64_t n_pts,
                          const float* ant_xyz, const float* c_ant, int32_t n_ant, const geraf_band* band,
                          int32_t flags, void* ws, size_t* ws_bytes, float* s_out, void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(n_pts >= 1 && n_ant >= 1, "render: need n_pts >= 1 and n_ant >= 1");
    REQUIRE(n_pts < (1ll << 31), "render: n_pts must be below 2^31");
    REQUIRE(band, "render: band must not be NULL");
    if (ws) REQUIRE(xyz && grad && w && t_eff && ant_xyz && c_ant && s_out, "render: null input or output");
    return render_impl(xyz, grad, w, t_eff, n_pts, ant_xyz, c_ant, n_ant, band, flags, ws, ws_bytes, s_out,
                       S(stream));
}

geraf_status geraf_render_noalloc(const float* xyz, const float* grad, const float* w, const float* t_eff,
                                  int64_t n_pts, const float* ant_xyz, const float* c_ant, int32_t n_ant,
                                  const geraf_band* band, int32_t flags, float* s_out, void* stream) {
    REQUIRE(n_pts >= 1 && n_ant >= 1, "render_noalloc: need n_pts >= 1 and n_ant >= 1");
    REQUIRE(n_pts < (1ll << 31), "render_noalloc: n_pts must be below 2^31");
    REQUIRE(band, "render_noalloc: band must not be NULL");
    REQUIRE(xyz && grad && w && t_eff && ant_xyz && c_ant && s_out, "render_noalloc: null input or output");
    return render_noalloc_impl(xyz, grad, w, t_eff, n_pts, ant_xyz, c_ant, n_ant, band, flags, s_out, S(stream));
}

geraf_status geraf_render_backward(const float* xyz, const float* grad, const float* w, const float* t_eff,
                                   int64_t n_pts, const float* ant_xyz, const float* c_ant, int32_t n_ant,
                                   const geraf_band* band, int32_t flags, const float* g_s, void* ws,
                                   size_t* ws_bytes, float* d_w, float* d_teff, float* d_grad, void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(n_pts >= 1 && n_ant >= 1, "render_backward: need n_pts >= 1 and n_ant >= 1");
    REQUIRE(n_pts < (1ll << 31), "render_backward: n_pts must be below 2^31");
    REQUIRE(band, "render_backward: band must not be NULL");
    if (ws)
        REQUIRE(xyz && grad && w && t_eff && ant_xyz && c_ant && g_s && d_w && d_teff && d_grad,
                "render_backward: null input or output");
    return render_backward_impl(xyz, grad, w, t_eff, n_pts, ant_xyz, c_ant, n_ant, band, flags, g_s, ws, ws_bytes,
                                d_w, d_teff, d_grad, S(stream));
}

geraf_status geraf_filter(const float* s, const float* ant_xyz, int32_t n_ant, const geraf_band* band,
                          const float* vox_xyz, int64_t n_vox, const float* target, const float* mask, void* ws,
                          size_t* ws_bytes, float* P, float* M, double* loss, float* dloss_dP, void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(n_vox >= 1 && n_ant >= 1, "filter: need n_vox >= 1 and n_ant >= 1");
    REQUIRE(n_vox < (1ll << 31), "filter: n_vox must be below 2^31");
    REQUIRE(band, "filter: band must not be NULL");
    if (ws) REQUIRE(s && ant_xyz && vox_xyz && P && M, "filter: null input or output");
    return filter_impl(s, ant_xyz, n_ant, band, vox_xyz, n_vox, target, mask, ws, ws_bytes, P, M, loss, dloss_dP,
                       S(stream));
}

geraf_status geraf_filter_backward(const float* ant_xyz, int32_t n_ant, const geraf_band* band, const float* vox_xyz,
                                   int64_t n_vox, const float* M, const float* d_P, void* ws, size_t* ws_bytes,
                                   float* g_s, void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(n_vox >= 1 && n_ant >= 1, "filter_backward: need n_vox >= 1 and n_ant >= 1");
    REQUIRE(n_vox < (1ll << 31), "filter_backward: n_vox must be below 2^31");
    REQUIRE(band, "filter_backward: band must not be NULL");
    if (ws) REQUIRE(ant_xyz && vox_xyz && M && d_P && g_s, "filter_backward: null input or output");
    return filter_backward_impl(ant_xyz, n_ant, band, vox_xyz, n_vox, M, d_P, ws, ws_bytes, g_s, S(stream));
}

geraf_status geraf_masked_loss(const float* P, const float* target, float* history, int64_t n_vox, float t_hi,
                               float t_lo, void* ws, size_t* ws_bytes, double* loss, float* dloss_dP, float* mask,
                               void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(n_vox >= 1 && n_vox < (1ll << 31), "masked_loss: need 1 <= n_vox < 2^31");
    if (ws) REQUIRE(P && target && history && loss, "masked_loss: null input or output");
    return masked_loss_impl(P, target, history, n_vox, t_hi, t_lo, ws, ws_bytes, loss, dloss_dP, mask, S(stream));
}

geraf_status geraf_chebyshev_order(const float* xyz, int64_t n, const float* ant_xyz, int32_t n_ant,
                                   const geraf_band* band, void* ws, size_t* ws_bytes, int32_t* order,
                                   void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(n >= 1 && n_ant >= 1, "chebyshev_order: need n >= 1 and n_ant >= 1");
    REQUIRE(n < (1ll << 31), "chebyshev_order: n must be below 2^31");
    REQUIRE(band, "chebyshev_order: band must not be NULL");
    if (ws) REQUIRE(xyz && ant_xyz && order, "chebyshev_order: null input or output");
    return chebyshev_order_impl(xyz, n, ant_xyz, n_ant, band, ws, ws_bytes, order, S(stream));
}

geraf_status geraf_chebyshev_work(const float* xyz, int64_t n, const float* ant_xyz, int32_t n_ant,
                                  const geraf_band* band, int32_t to_points, void* ws, size_t* ws_bytes,
                                  int32_t* orders, double* mean_orders, void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(n >= 1 && n_ant >= 1, "chebyshev_work: need n >= 1 and n_ant >= 1");
    REQUIRE(n < (1ll << 31), "chebyshev_work: n must be below 2^31");
    REQUIRE(band, "chebyshev_work: band must not be NULL");
    REQUIRE(to_points == 0 || to_points == 1, "chebyshev_work: to_points must be 0 or 1");
    if (ws) REQUIRE(xyz && ant_xyz && orders && mean_orders, "chebyshev_work: null input or output");
    return chebyshev_work_impl(xyz, n, ant_xyz, n_ant, band, to_points, ws, ws_bytes, orders, mean_orders,
                               S(stream));
}

geraf_status geraf_proposal_saved_bytes(const geraf_proposal* p, size_t* bytes) {
    REQUIRE(p && bytes, "proposal_saved_bytes: null argument");
    return proposal_saved_bytes(p, bytes);
}

geraf_status geraf_proposal_density(const geraf_proposal* p, float* logits, float* q, void* saved, size_t saved_bytes,
                                    void* stream) {
    REQUIRE(p && logits, "proposal_density: p and logits must not be NULL");
    return proposal_density_impl(p, logits, q, saved, saved_bytes, S(stream));
}

static geraf_status check_prop_grid(const geraf_grid* grid, const geraf_proposal* p) {
    REQUIRE(grid && p, "proposal: grid and p must not be NULL");
    for (int d = 0; d < 3; ++d) {
        REQUIRE(grid->n[d] > 0 && grid->pitch[d] > 0.0f, "proposal: bad grid");
        REQUIRE(p->g[d] > 0, "proposal: bad proposal grid");
    }
    REQUIRE(grid->n[0] % p->g[0] == 0 && grid->n[1] % p->g[1] == 0,
            "proposal: sample columns (%d x %d) must be multiples of the proposal grid (%d x %d)", grid->n[0],
            grid->n[1], p->g[0], p->g[1]);
    return GERAF_OK;
}

geraf_status geraf_sample_proposal(const geraf_grid* grid, const geraf_proposal* p, const float* q, uint64_t seed,
                                   uint64_t step, float* xyz, float* xyz_apr, int32_t* idx, void* stream) {
    geraf_status st = check_prop_grid(grid, p);
    if (st != GERAF_OK) return st;
    REQUIRE(q && xyz && idx, "sample_proposal: q, xyz and idx must not be NULL");
    REQUIRE((int64_t)grid->n[0] * grid->n[1] * p->depth < (1ll << 40), "sample_proposal: too many samples");
    REQUIRE(step < (1ull << 22), "sample_proposal: step must be below 2^22");
    return sample_proposal_impl(grid, p, q, seed, step, xyz, xyz_apr, idx, S(stream));
}

geraf_status geraf_sample_cells(const geraf_grid* grid, const geraf_proposal* p, const float* q, int32_t m,
                                int32_t r_max, int32_t dilate, uint64_t seed, uint64_t step, float* xyz,
                                float* xyz_apr, int32_t* idx, float* keep, void* ws, size_t* ws_bytes, void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    REQUIRE(grid && p, "sample_cells: grid and proposal must not be NULL");
    REQUIRE(grid->n[0] >= 1 && grid->n[1] >= 1 && grid->n[2] >= 1, "sample_cells: bad grid");
    REQUIRE(step < (1ull << 22), "sample_cells: step must be below 2^22");
    if (ws) REQUIRE(q && xyz && idx && keep, "sample_cells: null input or output");
    return sample_cells_impl(grid, p, q, m, r_max, dilate, seed, step, xyz, xyz_apr, idx, keep, ws, ws_bytes,
                             S(stream));
}

geraf_status geraf_sample_backward(const geraf_proposal* p, const geraf_grid* grid, int32_t n_z, const float* alpha,
                                   const float* T, const int32_t* idx, const float* logits, const void* saved,
                                   float* d_params, float* d_features, double* loss, void* ws, size_t* ws_bytes,
                                   void* stream) {
    geraf_status st = check_ws(ws, ws_bytes);
    if (st != GERAF_OK) return st;
    st = check_prop_grid(grid, p);
    if (st != GERAF_OK) return st;
    REQUIRE(n_z >= 1, "sample_backward: n_z must be >= 1");
    if (!idx) REQUIRE(n_z % p->g[2] == 0, "sample_backward: regular-grid depths %d not a multiple of G2 %d", n_z, p->g[2]);
    if (ws) REQUIRE(alpha && T && logits && saved && d_params && d_features, "sample_backward: null input or output");
    return sample_backward_impl(p, grid, n_z, alpha, T, idx, logits, saved, d_params, d_features, loss, ws, ws_bytes,
                                S(stream));
}

}  // extern "C"
