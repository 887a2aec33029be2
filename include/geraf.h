/*
 * geraf.h — C ABI of the GB300 (sm_103a) lensless RF volumetric rendering
 * hot path of GeRaF ("GeRaF: Neural Geometry Reconstruction from Radio
 * Frequency Signals", arXiv 2605.29097).
 *
 * Conventions shared by every call
 * --------------------------------
 * - All array arguments are DEVICE pointers owned by the caller, who also
 *   allocates every output. Nothing is allocated inside a call except where a
 *   call says so; scratch memory is the caller's workspace `ws`.
 * - Workspace protocol: calls taking (void* ws, size_t* ws_bytes) write the
 *   bytes they need to *ws_bytes and return GERAF_OK without launching when
 *   ws == NULL; otherwise *ws_bytes must hold at least that many bytes
 *   (GERAF_ERR_WORKSPACE if not). `ws` must be 256-byte aligned.
 * - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *   Every call is asynchronous on that stream; none synchronises the device.
 * - Layouts: FP32 structure-of-arrays. Positions/gradients are [3][n]
 *   (all x, then all y, then all z). Complex arrays are interleaved FP32
 *   (re, im) pairs, row-major [n_ant][n_f] for signals.
 * - Sample points are depth-major: point index = k * n_ray + ray, ray index =
 *   iy * nx + ix of the primary column.
 * - Every call returns a geraf_status; on error nothing was launched (argument
 *   errors) or the CUDA error is reported (GERAF_ERR_CUDA).
 *   geraf_last_error_string() gives a one-line description of the last error
 *   on the calling thread. No exception crosses the ABI.
 * - Results are deterministic: no floating-point atomics; split reductions are
 *   summed in a fixed order (in FP64, or in FP32 with Kahan compensation).
 */
#ifndef GERAF_H
#define GERAF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GERAF_OK = 0,
    GERAF_ERR_INVALID_ARG = 1,   /* null pointer, bad size or mode         */
    GERAF_ERR_ALIGNMENT = 2,     /* pointer not aligned as documented      */
    GERAF_ERR_CUDA = 3,          /* a CUDA runtime call or launch failed   */
    GERAF_ERR_WORKSPACE = 4,     /* workspace smaller than required        */
    GERAF_ERR_TIMEOUT = 5,       /* a bounded device-side wait ran out     */
    GERAF_ERR_UNSUPPORTED = 6    /* size or option outside the supported set */
} geraf_status;

/* Sample grid (section 6 "Primary Ray"): n[0] x n[1] primary columns parallel
 * to +z over the face of an axis-aligned box, n[2] depths per column. Cell
 * (ix, iy, k) spans lo + (i, i+1) * pitch on each axis. aperture_z is the
 * plane (z) of the primary rays' start points x_apr. */
typedef struct {
    float lo[3];
    float pitch[3];
    int32_t n[3];
    float aperture_z;
} geraf_grid;

/* Stepped frequencies f_n = f0 + n * df, n = 0 .. n_f-1 (section 3, Eq. fmcw:
 * FMCW sample n of a chirp with slope k is the frequency f + k t_n). FP64.
 * 1 <= n_f <= 1024, f0 > 0, df >= 0.
 * `method` picks how the four phasor sums (render, filter and their
 * adjoints) step across the bins; all give the same sums within FP32
 * rounding:
 *   GERAF_PHASOR_RECURRENCE: exact phasor per bin by angle-addition
 *     recurrence, re-seeded from a sincos every 32 bins;
 *   GERAF_PHASOR_CHEBYSHEV: the bin phase about the band's centre f_c,
 *     exp(-j 2 pi (n - (n_f - 1) / 2) df 2r/c), expanded in Chebyshev
 *     polynomials of the range (Jacobi-Anger, terms kept until the Bessel
 *     tail is below 1e-7, under the FP32 rounding of the sums), each run of
 *     consecutive points against each block of 128 antennas (taken in a
 *     spatial order of their positions) with its own half range, each
 *     antenna's interval centred on that antenna's own ranges, so the work
 *     per (point, antenna) pair follows the
 *     order instead of n_f; when the whole call's order K would exceed 64
 *     the recurrence runs instead (decided on the device;
 *     geraf_chebyshev_order reports the choice, geraf_chebyshev_work the
 *     orders evaluated);
 *   GERAF_PHASOR_AUTO (0): Chebyshev for n_f >= 64, recurrence below. */
typedef struct {
    double f0;
    double df;
    int32_t n_f;
    int32_t method;
} geraf_band;

enum { GERAF_PHASOR_AUTO = 0, GERAF_PHASOR_RECURRENCE = 1, GERAF_PHASOR_CHEBYSHEV = 2 };

enum { GERAF_SAMPLE_UNIFORM = 0, GERAF_SAMPLE_STRATIFIED = 1 };
enum { GERAF_FIELD_ANALYTIC = 0, GERAF_FIELD_MLP = 1 };
enum { GERAF_PREC_FP32 = 0, GERAF_PREC_BF16 = 1 };
enum { GERAF_PRIM_SPHERE = 0, GERAF_PRIM_BOX = 1, GERAF_PRIM_ELLIPSOID = 2, GERAF_PRIM_HALFSPACE = 3 };
enum { GERAF_RENDER_DIRECTIONAL = 1 };

/* Field description for geraf_fields.
 * ANALYTIC: `prims` points to n_prims records of 8 FP32 values
 *   (kind, a, c[3], p[3]); sphere p[0] = radius, box p = half extents,
 *   ellipsoid p = radii (first-order distance (|d/R| - 1) min R), half-space
 *   c = point on the plane, p = unit normal towards free space. The scene SDF
 *   is the minimum over primitives; G and a are the minimiser's.
 * MLP: `params` points to the packed FP32 parameters
 *   [W1 b1 ... W_nh b_nh W_head b_head], W row-major [out][in]; input is the
 *   positional encoding (section 9.3) of (x - center)/half with n_levels
 *   octaves (6 n_levels features: 6k+d = sin(2^k pi x_d), 6k+3+d = cos),
 *   n_hidden softplus(beta) layers of `width`, head [f, a_logit],
 *   a = sigmoid(a_logit).
 *   refl_hidden > 0 selects the paper's two separate networks (App. C
 *   "Training Setup"; section 5.2 "Signal representation"): an SDF network
 *   (n_hidden layers of `width`, head [f]) and a reflectivity network
 *   (refl_hidden layers of refl_width, head [a_logit]) on the same encoding,
 *   params packed [SDF network | reflectivity network], each as above.
 *   One 128-wide trunk (refl_hidden = 0, width = 128) runs the fused kernels
 *   in FP32 or BF16; every other shape runs layer by layer, in FP32 on CUDA
 *   cores (widths a multiple of 32 up to 1024) or in BF16 on the tensor cores
 *   (widths a multiple of 64 up to 256), up to 16 layers per network; it
 *   keeps its layer activations in `saved` (so `saved` is required even
 *   without a backward pass) and must be called with grad and refl for a
 *   backward pass to follow. BF16 means the BF16 network reading: weights and
 *   every hidden layer's inputs rounded to bfloat16, FP32 accumulation, bias,
 *   nonlinearity and head in FP32, straight-through adjoint.
 *   Zero-initialised trailing fields keep the single-trunk form. */
typedef struct {
    int32_t kind;
    const float* prims;
    int32_t n_prims;
    const float* params;
    int32_t n_levels;
    int32_t width;
    int32_t n_hidden;
    float beta;
    float center[3];
    float half;
    int32_t precision;
    int32_t refl_hidden;     /* 0: one trunk with head [f, a_logit] */
    int32_t refl_width;
} geraf_field_desc;

const char* geraf_last_error_string(void);
int32_t geraf_version(void);

/*
 * geraf_poll_device_error — synchronises `stream`, then reads and clears the
 * device error word of the current device. Returns GERAF_ERR_TIMEOUT when a
 * kernel gave up a bounded wait (a TMA copy or barrier that did not complete
 * within ~2 s; the kernel then left without writing its outputs), GERAF_OK
 * otherwise, GERAF_ERR_CUDA when synchronisation fails.
 */
geraf_status geraf_poll_device_error(void* stream);

/*
 * geraf_check_bounded_wait — self-test of the failure path every TMA kernel
 * uses (not in the paper): one CTA waits on a shared-memory mbarrier that
 * nothing arrives at, gives up after about limit_ns nanoseconds (1 us .. 1 s),
 * records the timeout in the device error word and returns. The next
 * geraf_poll_device_error on the same device then reports GERAF_ERR_TIMEOUT and
 * clears the word; the context stays usable. Asynchronous on `stream`.
 * Errors: INVALID_ARG for a limit outside the range, CUDA for launch failures.
 */
geraf_status geraf_check_bounded_wait(uint64_t limit_ns, void* stream);

/*
 * geraf_sample — lensless sampling (section 6 "Primary Ray"; section 4 step 1).
 * Writes n_pts = n[0]*n[1]*n[2] points xyz [3][n_pts] (depth-major) and the
 * n_ray = n[0]*n[1] primary-ray start points xyz_apr [3][n_ray] = (x, y,
 * aperture_z). UNIFORM: cell centres. STRATIFIED: ray start jittered once per
 * column (x, y) and depth jittered per point, U = (SplitMix64 output number
 * (step<<42 | stream<<40 | index) of `seed`) >> 11 times 2^-53, streams
 * 0 = x (index ray), 1 = y (index ray), 2 = z (index point). Each coordinate
 * is float(lo + (i + U) * pitch) evaluated in FP64 with one rounding per
 * operation, so results are bit-exact with any IEEE implementation.
 * Errors: INVALID_ARG for null outputs, non-positive n or pitch, index space
 * above 2^40 points or step >= 2^22.
 */
geraf_status geraf_sample(const geraf_grid* grid, int32_t mode, uint64_t seed, uint64_t step,
                          float* xyz, float* xyz_apr, void* stream);

/*
 * geraf_fields — SDF f, its gradient G = grad f (section 5.2: the normal is
 * the SDF gradient) and reflectiveness a at n points xyz [3][n].
 * sdf [n], grad [3][n], refl [n] are outputs (grad and refl may be NULL for
 * the ray-origin evaluations that need f only).
 * MLP fields need `saved` (activations kept for the backward pass) of
 * geraf_fields_saved_bytes() bytes, or NULL when no backward pass follows.
 * Errors: INVALID_ARG (null/bad sizes; `saved` NULL for a layer-by-layer network), UNSUPPORTED (shape),
 * WORKSPACE (saved too small).
 */
geraf_status geraf_fields_saved_bytes(const geraf_field_desc* desc, int64_t n, size_t* bytes);
geraf_status geraf_fields(const geraf_field_desc* desc, const float* xyz, int64_t n,
                          float* sdf, float* grad, float* refl, void* saved, size_t saved_bytes,
                          void* stream);

/*
 * geraf_fields_backward — adjoint of the MLP fields (value, the three
 * gradient tangents and the reflectiveness head) for upstream d_sdf [n],
 * d_grad [3][n], d_refl [n] (any may be NULL = zero). Writes the parameter
 * gradient d_params (same packed layout as params, overwritten, not
 * accumulated). Needs the `saved` buffer of the matching geraf_fields call and
 * a workspace (query with ws == NULL).
 */
geraf_status geraf_fields_backward(const geraf_field_desc* desc, const float* xyz, int64_t n,
                                   const void* saved, const float* d_sdf, const float* d_grad,
                                   const float* d_refl, float* d_params,
                                   void* ws, size_t* ws_bytes, void* stream);

/*
 * geraf_blend — lensless alpha blending (section 5.2 "Discretization",
 * section 6 "Lensless Alpha Blending", App. B).
 * Inputs: sdf, refl [n_ray*n_z] depth-major; sdf_apr [n_ray] = f(x_apr);
 * sdf_ant [n_ant] = f at the antennas; sharpness s > 0 of the logistic CDF
 * Phi_s(x) = 1/(1+exp(-s x)); a_tx = A'_tx.
 * Outputs [n_ray*n_z]: alpha_k = max((Phi(f_k)-Phi(f_{k+1}))/Phi(f_k), 0)
 * (0 at the last depth), T_k = prod_{m<k}(1-alpha_m), w_k = a_k alpha_k A'_tx,
 * t_eff_k = T_k + Phi_s(f(x_apr)); c_ant [n_ant] = Phi_s(f(x_ant)).
 * Antenna i then sees T' = clamp(t_eff - c_ant_i, 0, 1) (App. B.2 integration;
 * the origin terms carry no gradient, section 6).
 * keep [n_ray*n_z] (NULL = all ones) multiplies w: a sample with keep = 0
 * still closes the interval of the sample before it (its f enters that
 * alpha) and its own alpha still attenuates T, but it reflects nothing (the
 * run-closing and padding samples of geraf_sample_cells).
 */
geraf_status geraf_blend(const float* sdf, const float* refl, int32_t n_ray, int32_t n_z,
                         const float* sdf_apr, const float* sdf_ant, int32_t n_ant,
                         float s, float a_tx,
                         float* alpha, float* T, float* w, float* t_eff, float* c_ant, const float* keep,
                         void* stream);

/*
 * geraf_blend_backward — adjoint of geraf_blend for upstream d_w, d_teff
 * [n_ray*n_z] (either may be NULL = zero), with the forward's keep (or NULL).
 * Writes d_sdf, d_refl [n_ray*n_z] and d_scalars[2] = {dL/ds, dL/dA'_tx}
 * (device, overwritten).
 */
geraf_status geraf_blend_backward(const float* sdf, const float* refl, const float* alpha,
                                  const float* T, int32_t n_ray, int32_t n_z, float s, float a_tx,
                                  const float* d_w, const float* d_teff,
                                  float* d_sdf, float* d_refl, float* d_scalars, const float* keep,
                                  void* ws, size_t* ws_bytes, void* stream);

/*
 * geraf_render — signal tracing (section 5.1, Eq. ref_sim; App. A.5-A.6,
 * Algorithm 2 [1]) with the amplitude of Eq. signal_amp_tracing:
 *   s(i, n) = sum_j A_ij exp(-j 2 pi f_n tau_ij),  tau_ij = 2 |x_j - a_i| / c,
 *   A_ij = w_j T'_ij^2 gamma_ij D_ij,  gamma = 1/(4 pi r)^2,
 *   T'_ij = clamp(t_eff_j - c_ant_i, 0, 1),
 *   D_ij = max(0, 2 (n_j . w_ij)^2 - 1) with n_j = G_j/|G_j| (monostatic
 *   shifted-Lambertian factor, section 3; D = 1 when G_j = 0 or without
 *   GERAF_RENDER_DIRECTIONAL in flags).
 * Inputs: xyz, grad [3][n_pts]; w, t_eff [n_pts]; ant_xyz [3][n_ant];
 * c_ant [n_ant]; band. Output s_out [n_ant][n_f] complex (overwritten).
 * Points must not coincide with antennas (r = 0 is clamped, result then
 * meaningless). Workspace holds the packed point tiles and split partials.
 */
geraf_status geraf_render(const float* xyz, const float* grad, const float* w, const float* t_eff,
                          int64_t n_pts, const float* ant_xyz, const float* c_ant, int32_t n_ant,
                          const geraf_band* band, int32_t flags,
                          void* ws, size_t* ws_bytes, float* s_out, void* stream);

/*
 * geraf_render_noalloc — the signal tracing of geraf_render, for callers
 * that cannot allocate device memory themselves (for example a plug-in whose
 * host application owns every device allocation, or code that runs where the
 * application forbids new allocations): it takes no workspace and allocates
 * nothing. The paper has no counterpart; this is an interface convenience.
 * Its scratch is one static device array of 32 MiB inside this library, held
 * by every GPU that loads the library until the process exits. The first call
 * on a device looks up that array's device address (once per device, with
 * the device current); make that first call before any stream capture.
 * All calls share the array: calls that overlap on the GPU (on different
 * streams or from different host threads) race and give undefined results.
 * Inputs that need more than 32 MiB of scratch (the packed points, 48 bytes
 * each, plus at least one n_ant x 32*ceil(n_f/32) complex partial) are
 * rejected with GERAF_ERR_UNSUPPORTED; use geraf_render for them. It always
 * steps across the bins by the per-bin recurrence, whatever band->method asks
 * (the Chebyshev form's tables would not fit the static array), so at 64 bins
 * and more it is several times slower than geraf_render's default. Results
 * match geraf_render to FP32 rounding (the split of the point sum may differ).
 */
geraf_status geraf_render_noalloc(const float* xyz, const float* grad, const float* w, const float* t_eff,
                                  int64_t n_pts, const float* ant_xyz, const float* c_ant, int32_t n_ant,
                                  const geraf_band* band, int32_t flags, float* s_out, void* stream);

/*
 * geraf_render_backward — adjoint of geraf_render (App. A.5, Algorithm 2
 * [2]) for g_s = dL/dRe s + j dL/dIm s [n_ant][n_f] complex:
 *   q_ij = sum_n Re(conj(g_in) exp(-j 2 pi f_n tau_ij)),
 * then d_w_j = sum_i T'^2 gamma D q, d_teff_j = sum_i w 2 T' [0<=t_eff-c_ant<=1]
 * gamma D q, d_grad_j = sum_i w T'^2 gamma q dD/dG. Outputs overwritten.
 */
geraf_status geraf_render_backward(const float* xyz, const float* grad, const float* w,
                                   const float* t_eff, int64_t n_pts, const float* ant_xyz,
                                   const float* c_ant, int32_t n_ant, const geraf_band* band,
                                   int32_t flags, const float* g_s,
                                   void* ws, size_t* ws_bytes,
                                   float* d_w, float* d_teff, float* d_grad, void* stream);

/*
 * geraf_filter — matched filter heatmap (section 3, Eq. mf-sm; App. A.5,
 * Algorithm 1 [1]) and the L2 heatmap loss (section 4 step 5):
 *   M_v = sum_i sum_n s(i, n) exp(+j 2 pi f_n tau_iv),  P_v = |M_v|,
 *   loss = sum_v m_v (P_v - P*_v)^2,  dloss_dP_v = 2 m_v (P_v - P*_v).
 * Inputs: s [n_ant][n_f] complex, ant_xyz [3][n_ant], band, vox_xyz
 * [3][n_vox]; target P* [n_vox] and mask m [n_vox] optional (NULL mask = 1).
 * Outputs: P [n_vox], M [n_vox] complex (kept for the backward pass);
 * loss (one double, device) and dloss_dP [n_vox] only when target != NULL
 * (either output pointer may be NULL).
 */
geraf_status geraf_filter(const float* s, const float* ant_xyz, int32_t n_ant, const geraf_band* band,
                          const float* vox_xyz, int64_t n_vox, const float* target, const float* mask,
                          void* ws, size_t* ws_bytes,
                          float* P, float* M, double* loss, float* dloss_dP, void* stream);

/*
 * geraf_filter_backward — adjoint of P = |M(s)| (App. A.5, Algorithm 1 [2])
 * for upstream d_P [n_vox]:
 *   g(i, n) = sum_v d_P_v (M_v/|M_v|) exp(-j 2 pi f_n tau_iv)
 * (the printed gradient omits the M_v/|M_v| factor; a voxel with M_v = 0
 * contributes 0). Output g_s [n_ant][n_f] complex (overwritten).
 */
geraf_status geraf_filter_backward(const float* ant_xyz, int32_t n_ant, const geraf_band* band,
                                   const float* vox_xyz, int64_t n_vox, const float* M,
                                   const float* d_P, void* ws, size_t* ws_bytes,
                                   float* g_s, void* stream);

/*
 * geraf_masked_loss — dynamic loss masking (section 6, "Dynamic loss
 * masking") with the L2 heatmap loss (section 4, step 5): a voxel whose
 * matched-filter response was high in an earlier call (history_v >= t_hi)
 * but is low now (P_v < t_lo) is left out of the loss, m_v = 0, else m_v = 1;
 *   loss = sum_v m_v (P_v - P*_v)^2,  dloss_dP_v = 2 m_v (P_v - P*_v),
 * and then history_v = max(history_v, P_v) in place (a fresh history is all
 * zeros). The paper gives no thresholds: t_hi and t_lo are absolute powers
 * chosen by the caller, compared in FP32.
 * P, target, history [n_vox] FP32 device arrays; loss: one double (device,
 * overwritten); dloss_dP and mask [n_vox] (either may be NULL). The loss is
 * summed in FP64 in a fixed order. ws: ws == NULL queries *ws_bytes.
 */
geraf_status geraf_masked_loss(const float* P, const float* target, float* history, int64_t n_vox, float t_hi,
                               float t_lo, void* ws, size_t* ws_bytes, double* loss, float* dloss_dP, float* mask,
                               void* stream);

/*
 * geraf_chebyshev_order — the Chebyshev order K that the phasor sums use for
 * points (or voxels) xyz [3][n] against ant_xyz [3][n_ant] over `band`
 * (band->method honoured): *order = K (2..64) when the Chebyshev form runs,
 * 0 when the recurrence runs (method RECURRENCE, AUTO with n_f < 64, or an
 * order above 64). Runs the same device-side plan as the sums (the largest
 * half range over the antennas from the points' bounding box, each antenna's
 * interval about its own centre; the largest Bessel argument at the bins
 * (n_f - 1) / 2 from the band's centre; Bessel tail below 1e-7),
 * then waits for the stream: synchronous. The paper has no counterpart; this
 * reports the cost model of a call. ws: ws == NULL queries *ws_bytes.
 */
geraf_status geraf_chebyshev_order(const float* xyz, int64_t n, const float* ant_xyz, int32_t n_ant,
                                   const geraf_band* band, void* ws, size_t* ws_bytes, int32_t* order,
                                   void* stream);

/*
 * geraf_chebyshev_work — the orders one Chebyshev phasor call evaluates for
 * points (or voxels) xyz [3][n] against ant_xyz [3][n_ant] over `band`.
 * to_points = 0: the to-bins direction (geraf_render on points,
 * geraf_filter_backward on voxels), which expands each split of consecutive
 * point tiles (against each block of 128 antennas in their spatial order,
 * when the split is large enough) over its own range interval; to_points = 1:
 * the to-points direction (geraf_filter, geraf_render_backward), which
 * expands each group of consecutive points (at least 2048) against each
 * antenna block over its own interval. Outputs:
 * orders[0] = the whole set's order K (0: the recurrence runs; then all
 * outputs are 0), orders[1] = the largest part order, orders[2] = the orders
 * compiled into the kernel instance that runs (24, 32 or 64);
 * *mean_orders = the orders evaluated per (point, antenna) pair, averaged
 * over all pairs (in the 24- and 32-order instances each part's order rounded
 * up to even, at least 8; in the 64-order instance 32 plus the part's own
 * orders beyond 32 in blocks of 8). Runs the same device
 * plans as the sums, then waits for the stream: synchronous. The paper has no
 * counterpart; this reports the cost model of a call. ws: ws == NULL queries
 * *ws_bytes. GERAF_ERR_INVALID_ARG for n < 1, n >= 2^31, n_ant < 1, a NULL
 * band, or to_points not 0 or 1.
 */
geraf_status geraf_chebyshev_work(const float* xyz, int64_t n, const float* ant_xyz, int32_t n_ant,
                                  const geraf_band* band, int32_t to_points, void* ws, size_t* ws_bytes,
                                  int32_t* orders, double* mean_orders, void* stream);

/*
 * Learned proposal sampler (the paper is silent on it; it cuts the number of
 * lensless samples per step). A G0 x G1 x G2 grid of FP16 features over the
 * sample cube (cell index (gz*G1 + gy)*G0 + gx, features [n_cells][feat])
 * feeds a softplus(beta) MLP (n_hidden layers of `width`, one output logit;
 * packed FP32 params [W1 b1 ... W_out b_out], W row-major [out][in]). Per grid
 * column, q = (1 - eps) softmax(logits over gz) + eps / G2. A fine primary
 * column (ix, iy) of the sample grid uses grid column (ix*G0/nx, iy*G1/ny)
 * and draws `depth` depth samples by inverse CDF (see geraf_sample_proposal).
 */
typedef struct {
    const void* features;   /* FP16 [n_cells][feat], device */
    const float* params;    /* FP32 packed MLP parameters, device */
    int32_t g[3];           /* G0, G1, G2 (2 <= G2 <= 256) */
    int32_t feat;           /* 1 .. 16 */
    int32_t width;          /* 1 .. 64 */
    int32_t n_hidden;       /* 1 .. 4 */
    float beta;             /* softplus sharpness */
    float eps;              /* uniform floor of q, 0 <= eps < 1 */
    int32_t depth;          /* samples per primary column, 1 .. 256 */
} geraf_proposal;

/*
 * geraf_proposal_density — logits [n_cells] of every grid cell and (q != NULL)
 * the per-column depth distribution q [n_cells] (same cell order). `saved`
 * (geraf_proposal_saved_bytes, may be NULL) keeps the pre-activations for
 * geraf_sample_backward.
 */
geraf_status geraf_proposal_saved_bytes(const geraf_proposal* p, size_t* bytes);
geraf_status geraf_proposal_density(const geraf_proposal* p, float* logits, float* q, void* saved,
                                    size_t saved_bytes, void* stream);

/*
 * geraf_sample_proposal — lensless samples of `grid`'s n[0] x n[1] primary
 * columns, `depth` per column, drawn from q (section 6 "Primary Ray" with the
 * depths importance-sampled). Integer CDF per column: c_k = max(1,
 * floor(q_k 2^20)), C_{k+1} = C_k + c_k, W = C_G2; sample j: m_j = SplitMix64
 * output number (step<<42 | 3<<40 | ray*depth + j) of seed, shifted right by
 * 40 (24 bits); u_j = ((j<<24) + m_j) W / (depth<<24) (integer division);
 * cell k with C_k <= u_j < C_{k+1}; z = lo_z + (k + (u_j - C_k + 0.5)/c_k) *
 * pz_cell in FP64 with pz_cell = float(pitch_z n_z / G2), rounded to FP32.
 * The column's (x, y) are jittered as in STRATIFIED sampling. Outputs:
 * xyz [3][n_ray*depth] depth-major (samples sorted along every column),
 * xyz_apr [3][n_ray] (may be NULL), idx [n_ray*depth] = grid cell of each
 * sample. Bit-exact with any IEEE implementation given the same FP32 q.
 * Requires n[0] % G0 == 0 and n[1] % G1 == 0.
 */
geraf_status geraf_sample_proposal(const geraf_grid* grid, const geraf_proposal* p, const float* q,
                                   uint64_t seed, uint64_t step, float* xyz, float* xyz_apr, int32_t* idx,
                                   void* stream);

/*
 * geraf_sample_cells — lensless samples restricted to the depth cells the
 * proposal ranks highest (the task's learned sampler; the paper has none):
 * the grid's n[2] fine depths per column are grouped into the proposal's G2
 * cells of s = n[2] / G2 consecutive depths. Per grid column (the fine column
 * (ix, iy) uses (ix*G0/nx, iy*G1/ny)) the m cells ranked first are kept: by
 * the largest q within `dilate` cells of the cell (dilate = 0: its own q),
 * then by its own q, then the lower cell (FP32 q of geraf_proposal_density),
 * so that with dilate > 0 the neighbours of a peak, where the tails of its
 * weight lie, come before lone cells elsewhere. A fine
 * column's samples are exactly the STRATIFIED grid's own points in those
 * cells (geraf_sample with the same seed and step gives the same values bit
 * for bit), in depth order. After each run of consecutive kept cells (the
 * first r_max runs in depth order; not after the last cell) one more sample,
 * the first fine depth of the next cell, closes the run: the NeuS alpha of the
 * run's last sample then spans one fine interval, and the closing sample's own
 * alpha spans the skipped gap to the next kept sample (exactly the gap's
 * transmittance when f decreases through it). The column's n_out = m s +
 * r_max slots are filled with copies of its last sample (alpha 0). keep = 1
 * on kept-cell samples, 0 on closing and padding samples (pass it to
 * geraf_blend). Outputs (depth-major, n = n_ray * n_out): xyz [3][n],
 * xyz_apr [3][n_ray] (may be NULL), idx [n] = grid cell of each sample (the
 * next cell for a closing sample), keep [n]. Requires n[2] % G2 == 0,
 * n[0] % G0 == 0, n[1] % G1 == 0, 1 <= m <= G2, 0 <= r_max <= m,
 * 0 <= dilate < G2; a workspace
 * (per grid column table of n_out int32; ws == NULL queries *ws_bytes).
 * Deterministic and bit-exact with any IEEE implementation given the same q.
 */
geraf_status geraf_sample_cells(const geraf_grid* grid, const geraf_proposal* p, const float* q, int32_t m,
                                int32_t r_max, int32_t dilate, uint64_t seed, uint64_t step, float* xyz,
                                float* xyz_apr, int32_t* idx, float* keep, void* ws, size_t* ws_bytes, void* stream);

/*
 * geraf_sample_backward — online training signal of the proposal from the
 * blended weights of a render: target p per grid column = normalised
 * histogram of T*alpha (geraf_blend outputs, [n_z][n_ray] of `grid`) over the
 * column's cells; loss = sum over columns with weight of KL(p || q).
 * idx = the sample cells of geraf_sample_proposal, or NULL for samples of the
 * regular grid (n_z = grid.n[2], which must be a multiple of G2). Writes
 * d_params (packed like params), d_features (FP32 [n_cells][feat]) and loss
 * (one double, may be NULL). Needs `logits` and `saved` of
 * geraf_proposal_density and a workspace.
 */
geraf_status geraf_sample_backward(const geraf_proposal* p, const geraf_grid* grid, int32_t n_z,
                                   const float* alpha, const float* T, const int32_t* idx,
                                   const float* logits, const void* saved, float* d_params,
                                   float* d_features, double* loss, void* ws, size_t* ws_bytes,
                                   void* stream);

#ifdef __cplusplus
}
#endif
#endif /* GERAF_H */
