// Learned proposal sampler: a coarse G0 x G1 x G2 grid of FP16 features with a
// small softplus MLP gives a logit per cell; per grid column the depth
// distribution is q = (1 - eps) softmax(logits) + eps / G2. Lensless samples
// of a fine primary column are drawn by inverse CDF from an integer CDF of q
// (bit-exact), so the network concentrates the column's depth samples where
// the blended weights are. The network is trained online on those weights:
// loss = sum over grid columns of KL(p || q), p = the normalised histogram of
// the geometric weights T alpha of the rendered samples in the column's cells.
#include <cuda_fp16.h>
#include <math.h>

#include "common.cuh"

namespace geraf {

namespace {

constexpr int PW = 64;        // maximum hidden width (kernels use fixed 64-wide registers)
constexpr int PF = 16;        // maximum feature dimension
constexpr int PNH = 4;        // maximum hidden layers
constexpr int PBT = 128;      // cells per backward tile / threads per CTA
constexpr int PWS = PW + 1;   // row stride of the backward's per-cell shared rows (thread = row: no bank conflicts)

struct PropGeom {
    int G0, G1, G2, F, W, NH, D;
    float beta, eps;
    int64_t n_cells, n_params;
    int off_w[PNH + 1], off_b[PNH + 1], k_in[PNH + 1], n_out[PNH + 1];
};

bool make_prop(const geraf_proposal* p, PropGeom* g) {
    if (!p || !p->features || !p->params) {
        set_error("proposal: features and params must not be NULL");
        return false;
    }
    if (p->g[0] < 1 || p->g[1] < 1 || p->g[2] < 2 || p->g[2] > 256 || p->feat < 1 || p->feat > PF ||
        p->width < 1 || p->width > PW || p->n_hidden < 1 || p->n_hidden > PNH || p->depth < 1 || p->depth > 256 ||
        !(p->eps >= 0.0f && p->eps < 1.0f)) {
        set_error("proposal: need G2 in [2, 256], 1 <= feat <= 16, 1 <= width <= 64, 1 <= n_hidden <= 4, "
                  "1 <= depth <= 256, 0 <= eps < 1");
        return false;
    }
    g->G0 = p->g[0]; g->G1 = p->g[1]; g->G2 = p->g[2];
    g->F = p->feat; g->W = p->width; g->NH = p->n_hidden; g->D = p->depth;
    g->beta = p->beta; g->eps = p->eps;
    g->n_cells = (int64_t)g->G0 * g->G1 * g->G2;
    int off = 0;
    for (int l = 0; l <= g->NH; ++l) {
        g->k_in[l] = l == 0 ? g->F : g->W;
        g->n_out[l] = l == g->NH ? 1 : g->W;
        g->off_w[l] = off; off += g->n_out[l] * g->k_in[l];
        g->off_b[l] = off; off += g->n_out[l];
    }
    g->n_params = off;
    return true;
}

__device__ __forceinline__ float sp_b(float h, float beta) {
    return fmaxf(h, 0.0f) + log1pf(expf(-beta * fabsf(h))) / beta;
}
__device__ __forceinline__ float sig(float x) { return 1.0f / (1.0f + expf(-x)); }

// ---------------------------------------------------------- network forward
// CTA = PFT cells; the hidden layers as register-tiled products: thread =
// (block of 8 cells, block of 8 units), 64 accumulators, the layer input held
// transposed in shared memory [k][cell] and the weights transposed [k][unit],
// so each input index k costs four 16-byte loads for 64 FMAs. Every unit's
// sum starts from its bias and adds the inputs in index order, as a plain
// dot product would. The output layer (one logit) runs per cell.
constexpr int PFT = 128;                 // cells per forward CTA
constexpr int PZS = PFT + 4;             // row stride of the transposed activations
static_assert(PW % 8 == 0 && PFT == 16 * 8, "forward tiling: 16 cell blocks x 8 unit blocks of 8");

size_t prop_forward_smem(const PropGeom& g) {
    return ((size_t)g.NH * PW * PW + (size_t)g.NH * PW + PW + 4 + (size_t)PW * PZS) * sizeof(float);
}

__global__ void __launch_bounds__(PFT) prop_forward_kernel(PropGeom g, const __half* __restrict__ feat,
                                                           const float* __restrict__ params,
                                                           float* __restrict__ logits, float* __restrict__ saved) {
    extern __shared__ __align__(16) float sm[];
    float* wt = sm;                                  // [NH][PW k][PW u], zero for u >= W or k >= K
    float* bs = wt + (size_t)g.NH * PW * PW;         // [NH][PW]
    float* wo = bs + g.NH * PW;                      // [PW] output weights, then the output bias
    float* zs = wo + PW + 4;                         // [PW k][PZS]: the layer input, transposed
    const int t = threadIdx.x;
    for (int i = t; i < g.NH * PW * PW; i += PFT) {
        const int l = i / (PW * PW), r = i - l * PW * PW, k = r / PW, u = r - k * PW;
        const int K = g.k_in[l];
        wt[i] = (u < g.W && k < K) ? params[g.off_w[l] + u * K + k] : 0.0f;
    }
    for (int i = t; i < g.NH * PW; i += PFT) {
        const int l = i / PW, u = i - l * PW;
        bs[i] = u < g.W ? params[g.off_b[l] + u] : 0.0f;
    }
    for (int i = t; i < PW; i += PFT) wo[i] = i < g.W ? params[g.off_w[g.NH] + i] : 0.0f;
    if (t == 0) wo[PW] = params[g.off_b[g.NH]];
    const int64_t c0 = (int64_t)blockIdx.x * PFT;
    {
        const int64_t c = min(c0 + t, g.n_cells - 1);
        for (int k = 0; k < g.F; ++k) zs[k * PZS + t] = __half2float(feat[c * g.F + k]);
    }
    __syncthreads();
    const int ci = t >> 3, ui = t & 7;               // cells 8 ci .. + 7, units 8 ui .. + 7
    for (int l = 0; l < g.NH; ++l) {
        const int K = g.k_in[l];
        const float* wl = wt + (size_t)l * PW * PW;
        float acc[8][8];
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const float b = bs[l * PW + 8 * ui + j];
#pragma unroll
            for (int i = 0; i < 8; ++i) acc[i][j] = b;
        }
        for (int k = 0; k < K; ++k) {
            const float4 z0 = *reinterpret_cast<const float4*>(zs + k * PZS + 8 * ci);
            const float4 z1 = *reinterpret_cast<const float4*>(zs + k * PZS + 8 * ci + 4);
            const float4 w0 = *reinterpret_cast<const float4*>(wl + k * PW + 8 * ui);
            const float4 w1 = *reinterpret_cast<const float4*>(wl + k * PW + 8 * ui + 4);
            const float zc[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
            const float wu[8] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(wu[j], zc[i], acc[i][j]);
        }
        __syncthreads();                              // every thread has read this layer's input
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const int u = 8 * ui + j;
            if (u >= g.W) continue;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int64_t c = c0 + 8 * ci + i;
                if (saved && c < g.n_cells) saved[((int64_t)l * g.W + u) * g.n_cells + c] = acc[i][j];
            }
            float4 v0, v1;
            v0.x = sp_b(acc[0][j], g.beta); v0.y = sp_b(acc[1][j], g.beta);
            v0.z = sp_b(acc[2][j], g.beta); v0.w = sp_b(acc[3][j], g.beta);
            v1.x = sp_b(acc[4][j], g.beta); v1.y = sp_b(acc[5][j], g.beta);
            v1.z = sp_b(acc[6][j], g.beta); v1.w = sp_b(acc[7][j], g.beta);
            *reinterpret_cast<float4*>(zs + u * PZS + 8 * ci) = v0;
            *reinterpret_cast<float4*>(zs + u * PZS + 8 * ci + 4) = v1;
        }
        __syncthreads();
    }
    const int64_t c = c0 + t;
    if (c < g.n_cells) {
        float a = wo[PW];
        for (int k = 0; k < g.W; ++k) a = fmaf(wo[k], zs[k * PZS + t], a);
        logits[c] = a;
    }
}

__global__ void prop_q_kernel(PropGeom g, const float* __restrict__ logits, float* __restrict__ q) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int plane = g.G0 * g.G1;
    if (col >= plane) return;
    double mx = -1e300;
    for (int k = 0; k < g.G2; ++k) mx = fmax(mx, (double)logits[(int64_t)k * plane + col]);
    double s = 0.0;
    for (int k = 0; k < g.G2; ++k) s += exp((double)logits[(int64_t)k * plane + col] - mx);
    for (int k = 0; k < g.G2; ++k) {
        const double e = exp((double)logits[(int64_t)k * plane + col] - mx) / s;
        q[(int64_t)k * plane + col] = (float)((1.0 - (double)g.eps) * e + (double)g.eps / g.G2);
    }
}

// ------------------------------------------------------------------ sampling
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ float grid_coord(float lo, int64_t i, double u, float pitch) {
    double t = __dadd_rn((double)i, u);
    t = __dmul_rn(t, (double)pitch);
    return __double2float_rn(__dadd_rn((double)lo, t));
}

__global__ void prop_sample_kernel(geraf_grid gr, PropGeom g, const float* __restrict__ q, uint64_t seed,
                                   uint64_t step, float pz_cell, float* __restrict__ xyz, float* __restrict__ apr,
                                   int32_t* __restrict__ idx) {
    const int64_t n_ray = (int64_t)gr.n[0] * gr.n[1];
    const int64_t ray = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (ray >= n_ray) return;
    const int64_t n = n_ray * g.D;
    const int64_t ix = ray % gr.n[0], iy = ray / gr.n[0];
    const int gx = (int)(ix * g.G0 / gr.n[0]), gy = (int)(iy * g.G1 / gr.n[1]);
    const int plane = g.G0 * g.G1;
    const int col = gy * g.G0 + gx;
    const uint64_t s0 = step << 42;
    const double ux = (double)(splitmix64(seed, s0 | (0ull << 40) | (uint64_t)ray) >> 11) * 0x1.0p-53;
    const double uy = (double)(splitmix64(seed, s0 | (1ull << 40) | (uint64_t)ray) >> 11) * 0x1.0p-53;
    const float x = grid_coord(gr.lo[0], ix, ux, gr.pitch[0]);
    const float y = grid_coord(gr.lo[1], iy, uy, gr.pitch[1]);
    if (apr) {
        apr[ray] = x;
        apr[n_ray + ray] = y;
        apr[2 * n_ray + ray] = gr.aperture_z;
    }
    // integer CDF weights c_k = max(1, floor(q_k 2^20)), total W
    uint64_t Wt = 0;
    for (int k = 0; k < g.G2; ++k) {
        const double ck = floor((double)q[(int64_t)k * plane + col] * 1048576.0);
        Wt += ck < 1.0 ? 1ull : (uint64_t)ck;
    }
    const uint64_t den = (uint64_t)g.D << 24;
    auto u_of = [&](int j) -> uint64_t {
        const uint64_t m = splitmix64(seed, s0 | (3ull << 40) | (uint64_t)(ray * g.D + j)) >> 40;
        return ((((uint64_t)j) << 24) + m) * Wt / den;
    };
    int j = 0;
    uint64_t uj = u_of(0);
    uint64_t C = 0;
    for (int k = 0; k < g.G2 && j < g.D; ++k) {
        const double ckd = floor((double)q[(int64_t)k * plane + col] * 1048576.0);
        const uint64_t ck = ckd < 1.0 ? 1ull : (uint64_t)ckd;
        while (j < g.D && uj < C + ck) {
            const double frac = __ddiv_rn(__dadd_rn((double)(uj - C), 0.5), (double)ck);
            const double zc = __dadd_rn((double)gr.lo[2], __dmul_rn(__dadd_rn((double)k, frac), (double)pz_cell));
            const int64_t p = (int64_t)j * n_ray + ray;
            xyz[p] = x;
            xyz[n + p] = y;
            xyz[2 * n + p] = __double2float_rn(zc);
            idx[p] = k * plane + col;
            ++j;
            if (j < g.D) uj = u_of(j);
        }
        C += ck;
    }
}

// ------------------------------------------------- samples of selected cells
// Depth cells of a grid column: the G2 cells of s = n_z / G2 consecutive fine
// depths each. Per grid column the m cells ranked first are kept (by the
// largest q within `dilate` cells, then the cell's own q, then the lower
// index); a fine column samples exactly the stratified grid's
// own points of those cells (bit for bit the points of a dense STRATIFIED
// geraf_sample with the same seed and step), so the kept part of the column is
// the dense render's; after each run of consecutive kept cells (the first
// r_max runs in depth order, and not past the last cell) one more sample, the
// first fine depth of the next cell, closes the run's last interval (its alpha
// uses f there, not at the next kept sample); that sample and the padding
// that fills the column's n_out = m s + r_max slots (copies of its last
// sample, so their alpha is 0) carry keep = 0.
// Table per grid column [n_out]: fine depth | (keep << 30).
__global__ void cells_select_kernel(PropGeom g, int s_fine, int m, int r_max, int dilate, int n_out,
                                    const float* __restrict__ q, int32_t* __restrict__ table) {
    __shared__ float qs[256];
    __shared__ float qd[256];
    __shared__ int sel[256];
    __shared__ int list[256];
    const int col = blockIdx.x, k = threadIdx.x;
    const int plane = g.G0 * g.G1;
    if (k < g.G2) qs[k] = q[(int64_t)k * plane + col];
    __syncthreads();
    // ranking key: the largest q within `dilate` cells (so the neighbours of a
    // peak come before a lone cell of smaller q), then the cell's own q, then
    // the lower cell index
    if (k < g.G2) {
        float v = qs[k];
        for (int j = max(0, k - dilate); j <= min(g.G2 - 1, k + dilate); ++j) v = fmaxf(v, qs[j]);
        qd[k] = v;
    }
    __syncthreads();
    int keep_k = 0;
    if (k < g.G2) {
        const float vd = qd[k], v = qs[k];
        int rank = 0;
        for (int j = 0; j < g.G2; ++j)
            rank += (qd[j] > vd || (qd[j] == vd && (qs[j] > v || (qs[j] == v && j < k)))) ? 1 : 0;
        keep_k = rank < m;
    }
    sel[k] = keep_k;
    __syncthreads();
    if (keep_k) {
        int pos = 0;
        for (int j = 0; j < k; ++j) pos += sel[j];
        list[pos] = k;
    }
    __syncthreads();
    if (k == 0) {
        int32_t* t = table + (int64_t)col * n_out;
        int o = 0, runs = 0;
        for (int i = 0; i < m; ++i) {
            const int c = list[i];
            for (int d = 0; d < s_fine; ++d) t[o++] = (c * s_fine + d) | (1 << 30);
            const bool run_end = i + 1 == m || list[i + 1] != c + 1;
            if (run_end && runs < r_max && c + 1 < g.G2) {
                t[o++] = (c + 1) * s_fine;
                ++runs;
            }
        }
        const int32_t last = t[o - 1] & ~(1 << 30);
        while (o < n_out) t[o++] = last;
    }
}

// thread = (fine column, slot): the slot's stratified grid point
__global__ void cells_sample_kernel(geraf_grid gr, PropGeom g, int s_fine, int n_out,
                                    const int32_t* __restrict__ table, uint64_t seed, uint64_t step,
                                    float* __restrict__ xyz, float* __restrict__ apr, int32_t* __restrict__ idx,
                                    float* __restrict__ keep) {
    const int64_t n_ray = (int64_t)gr.n[0] * gr.n[1];
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n_ray * n_out) return;
    const int64_t slot = e / n_ray, ray = e - slot * n_ray;
    const int64_t n = n_ray * n_out;
    const int64_t ix = ray % gr.n[0], iy = ray / gr.n[0];
    const int gx = (int)(ix * g.G0 / gr.n[0]), gy = (int)(iy * g.G1 / gr.n[1]);
    const int col = gy * g.G0 + gx;
    const int32_t code = table[(int64_t)col * n_out + slot];
    const int64_t kz = code & ~(1 << 30);
    const uint64_t s0 = step << 42;
    const double ux = (double)(splitmix64(seed, s0 | (0ull << 40) | (uint64_t)ray) >> 11) * 0x1.0p-53;
    const double uy = (double)(splitmix64(seed, s0 | (1ull << 40) | (uint64_t)ray) >> 11) * 0x1.0p-53;
    const double uz = (double)(splitmix64(seed, s0 | (2ull << 40) | (uint64_t)(kz * n_ray + ray)) >> 11) * 0x1.0p-53;
    const float x = grid_coord(gr.lo[0], ix, ux, gr.pitch[0]);
    const float y = grid_coord(gr.lo[1], iy, uy, gr.pitch[1]);
    xyz[e] = x;
    xyz[n + e] = y;
    xyz[2 * n + e] = grid_coord(gr.lo[2], kz, uz, gr.pitch[2]);
    idx[e] = (int32_t)((kz / s_fine) * (g.G0 * g.G1) + col);
    keep[e] = (code >> 30) & 1 ? 1.0f : 0.0f;
    if (apr && slot == 0) {
        apr[ray] = x;
        apr[n_ray + ray] = y;
        apr[2 * n_ray + ray] = gr.aperture_z;
    }
}

// --------------------------------------------------------- targets and loss
// histogram of T alpha over grid cells, gathered per cell in a fixed order
__global__ void prop_hist_kernel(geraf_grid gr, PropGeom g, int n_z, const float* __restrict__ alpha,
                                 const float* __restrict__ T, const int32_t* __restrict__ idx,
                                 double* __restrict__ hist) {
    const int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (cell >= g.n_cells) return;
    const int plane = g.G0 * g.G1;
    const int gz = (int)(cell / plane), rem = (int)(cell - (int64_t)gz * plane);
    const int gy = rem / g.G0, gx = rem - gy * g.G0;
    const int fx = gr.n[0] / g.G0, fy = gr.n[1] / g.G1;
    const int64_t n_ray = (int64_t)gr.n[0] * gr.n[1];
    double s = 0.0;
    for (int iy = gy * fy; iy < (gy + 1) * fy; ++iy)
        for (int ix = gx * fx; ix < (gx + 1) * fx; ++ix) {
            const int64_t ray = (int64_t)iy * gr.n[0] + ix;
            if (idx) {
                for (int j = 0; j < n_z; ++j) {
                    const int64_t p = (int64_t)j * n_ray + ray;
                    if (idx[p] == cell) s += (double)T[p] * (double)alpha[p];
                }
            } else {
                const int fz = n_z / g.G2;
                for (int j = gz * fz; j < (gz + 1) * fz; ++j) {
                    const int64_t p = (int64_t)j * n_ray + ray;
                    s += (double)T[p] * (double)alpha[p];
                }
            }
        }
    hist[cell] = s;
}

// The same histogram for samples with a cell index (idx): thread = grid
// column, one pass over the column's fine rays and their n_z samples, each
// sample added to the cell idx names (cells of other columns or out of range
// are skipped, as in prop_hist_kernel). A cell's sum runs in the same order
// (rays row by row, then depth) as prop_hist_kernel's, so the FP64 results
// are the same bit for bit, without every cell of a column rescanning the
// column's samples. Shared histogram [G2][blockDim] (conflict-free).
__global__ void prop_hist_cols_kernel(geraf_grid gr, PropGeom g, int n_z, const float* __restrict__ alpha,
                                      const float* __restrict__ T, const int32_t* __restrict__ idx,
                                      double* __restrict__ hist) {
    extern __shared__ double hs[];
    const int t = threadIdx.x, nb = blockDim.x;
    const int plane = g.G0 * g.G1;
    const int col = blockIdx.x * nb + t;
    for (int k = 0; k < g.G2; ++k) hs[k * nb + t] = 0.0;
    if (col >= plane) return;
    const int gy = col / g.G0, gx = col - gy * g.G0;
    const int fx = gr.n[0] / g.G0, fy = gr.n[1] / g.G1;
    const int64_t n_ray = (int64_t)gr.n[0] * gr.n[1];
    for (int iy = gy * fy; iy < (gy + 1) * fy; ++iy)
        for (int ix = gx * fx; ix < (gx + 1) * fx; ++ix) {
            const int64_t ray = (int64_t)iy * gr.n[0] + ix;
            for (int j = 0; j < n_z; ++j) {
                const int64_t p = (int64_t)j * n_ray + ray;
                const int64_t rel = (int64_t)idx[p] - col;
                if (rel < 0 || rel % plane != 0) continue;
                const int64_t gz = rel / plane;
                if (gz >= g.G2) continue;
                hs[gz * nb + t] += (double)T[p] * (double)alpha[p];
            }
        }
    for (int k = 0; k < g.G2; ++k) hist[(int64_t)k * plane + col] = hs[k * nb + t];
}

// per grid column: KL(p || q) and dL/dlogits (FP64 internally)
__global__ void prop_loss_kernel(PropGeom g, const float* __restrict__ logits, const double* __restrict__ hist,
                                 float* __restrict__ d_logits, double* __restrict__ col_loss) {
    const int col = blockIdx.x * blockDim.x + threadIdx.x;
    const int plane = g.G0 * g.G1;
    if (col >= plane) return;
    double tot = 0.0, mx = -1e300;
    for (int k = 0; k < g.G2; ++k) {
        tot += hist[(int64_t)k * plane + col];
        mx = fmax(mx, (double)logits[(int64_t)k * plane + col]);
    }
    if (!(tot > 0.0)) {
        for (int k = 0; k < g.G2; ++k) d_logits[(int64_t)k * plane + col] = 0.0f;
        col_loss[col] = 0.0;
        return;
    }
    double se = 0.0;
    for (int k = 0; k < g.G2; ++k) se += exp((double)logits[(int64_t)k * plane + col] - mx);
    const double eps = g.eps, a = 1.0 - eps;
    double kl = 0.0, rs = 0.0;
    for (int k = 0; k < g.G2; ++k) {
        const double sm = exp((double)logits[(int64_t)k * plane + col] - mx) / se;
        const double qk = a * sm + eps / g.G2;
        const double pk = hist[(int64_t)k * plane + col] / tot;
        if (pk > 0.0) kl += pk * (log(pk) - log(qk));
        rs += pk / qk * sm;
    }
    for (int k = 0; k < g.G2; ++k) {
        const double sm = exp((double)logits[(int64_t)k * plane + col] - mx) / se;
        const double qk = a * sm + eps / g.G2;
        const double pk = hist[(int64_t)k * plane + col] / tot;
        d_logits[(int64_t)k * plane + col] = (float)(a * sm * (-(pk / qk) + rs));
    }
    col_loss[col] = kl;
}

__global__ void sum_doubles_1(const double* __restrict__ x, int64_t n, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// --------------------------------------------------------- network adjoint
// Persistent CTAs over tiles of PBT cells. Thread = cell for the per-cell
// parts (pre-activation adjoint, input adjoint); thread = parameter entry for
// the weight-gradient sums over the tile's cells, accumulated in a per-CTA
// shared buffer (fixed order, no atomics).
__global__ void __launch_bounds__(PBT, 1) prop_backward_kernel(PropGeom g, const __half* __restrict__ feat,
                                                               const float* __restrict__ params,
                                                               const float* __restrict__ saved,
                                                               const float* __restrict__ d_logits,
                                                               float* __restrict__ d_feat,
                                                               float* __restrict__ partial) {
    extern __shared__ float sm[];
    float* sw = sm;                               // parameters
    float* gacc = sw + g.n_params;                // parameter gradient of this CTA
    float* hb = gacc + g.n_params;                // [PBT][PWS] pre-activation adjoint
    float* zi = hb + PBT * PWS;                    // [PBT][PWS] layer input
    float* dl = zi + PBT * PWS;                    // [PBT] d logits
    const int t = threadIdx.x;
    for (int i = t; i < g.n_params; i += PBT) {
        sw[i] = params[i];
        gacc[i] = 0.0f;
    }
    __syncthreads();
    const int W = g.W;
    // saved pre-activations of layer ll for the tile's cells into rows
    // dst[cell * PWS + unit], every load in flight (coalesced along the cells)
    auto stage = [&](float* dst, int ll, int64_t tile0) {
        const float* src = saved + (int64_t)ll * W * g.n_cells;
        for (int i = t; i < W * PBT; i += PBT) {
            const int u = i / PBT, q = i - u * PBT;
            const int64_t cq = min(tile0 + q, g.n_cells - 1);
            cp_async4(dst + q * PWS + u, src + (int64_t)u * g.n_cells + cq);
        }
    };
    for (int64_t tile = blockIdx.x; tile * PBT < g.n_cells; tile += gridDim.x) {
        const int64_t c = tile * PBT + t;
        const bool valid = c < g.n_cells;
        const int64_t cc = valid ? c : g.n_cells - 1;
        // output layer: zin = softplus(h_{NH-1}), hbar = d_logit
        stage(zi, g.NH - 1, tile * PBT);
        const float dlog = valid ? d_logits[cc] : 0.0f;
        dl[t] = dlog;
        float zb[PW];
        const float* Wo = sw + g.off_w[g.NH];
#pragma unroll
        for (int u = 0; u < PW; ++u) zb[u] = u < W ? Wo[u] * dlog : 0.0f;
        cp_async_wait_all();
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PW; ++u) zi[t * PWS + u] = u < W ? sp_b(zi[t * PWS + u], g.beta) : 0.0f;
        __syncthreads();
        for (int k = t; k < W; k += PBT) {
            float a = 0.0f;
            for (int q = 0; q < PBT; ++q) a = fmaf(dl[q], zi[q * PWS + k], a);
            gacc[g.off_w[g.NH] + k] += a;
        }
        if (t == 0) {
            float a = 0.0f;
            for (int q = 0; q < PBT; ++q) a += dl[q];
            gacc[g.off_b[g.NH]] += a;
        }
        __syncthreads();
        for (int l = g.NH - 1; l >= 0; --l) {
            const int K = g.k_in[l];
            // this layer's and (above the first) the layer below's
            // pre-activations, then, thread = cell, the pre-activation adjoint
            // and this layer's input in place
            stage(hb, l, tile * PBT);
            if (l > 0) stage(zi, l - 1, tile * PBT);
            cp_async_wait_all();
            __syncthreads();
#pragma unroll
            for (int u = 0; u < PW; ++u) {
                float v = 0.0f;
                if (u < W && valid) v = zb[u] * sig(g.beta * hb[t * PWS + u]);
                hb[t * PWS + u] = v;
            }
#pragma unroll
            for (int k = 0; k < PW; ++k) {
                float v = 0.0f;
                if (k < K) {
                    if (l > 0) v = sp_b(zi[t * PWS + k], g.beta);
                    else v = __half2float(feat[cc * g.F + k]);
                }
                zi[t * PWS + k] = v;
            }
            __syncthreads();
            // weight / bias gradient sums over the tile's cells: thread = block
            // of 4 units x 8 inputs, each entry summed over the cells in order
            {
                const int KB = (K + 7) / 8;
                for (int e = t; e < (W + 3) / 4 * KB; e += PBT) {
                    const int u0 = 4 * (e / KB), k0 = 8 * (e - (e / KB) * KB);
                    float acc[4][8];
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
                    for (int q = 0; q < PBT; ++q) {
                        float hv[4], zv[8];
#pragma unroll
                        for (int i = 0; i < 4; ++i) hv[i] = hb[q * PWS + min(u0 + i, PW - 1)];
#pragma unroll
                        for (int j = 0; j < 8; ++j) zv[j] = zi[q * PWS + min(k0 + j, PW - 1)];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(hv[i], zv[j], acc[i][j]);
                    }
#pragma unroll
                    for (int i = 0; i < 4; ++i)
#pragma unroll
                        for (int j = 0; j < 8; ++j)
                            if (u0 + i < W && k0 + j < K) gacc[g.off_w[l] + (u0 + i) * K + k0 + j] += acc[i][j];
                }
            }
            for (int u = t; u < W; u += PBT) {
                float a = 0.0f;
                for (int q = 0; q < PBT; ++q) a += hb[q * PWS + u];
                gacc[g.off_b[l] + u] += a;
            }
            // adjoint of the layer input, thread = cell
            const float* Wl = sw + g.off_w[l];
            float nz[PW];
#pragma unroll
            for (int k = 0; k < PW; ++k) nz[k] = 0.0f;
            for (int u = 0; u < W; ++u) {             // each nz[k] summed over u in order
                const float h = hb[t * PWS + u];
                const float* wr = Wl + u * K;
#pragma unroll
                for (int k = 0; k < PW; ++k)
                    if (k < K) nz[k] = fmaf(wr[k], h, nz[k]);
            }
            if (l == 0 && valid) {
                for (int k = 0; k < g.F; ++k) d_feat[c * g.F + k] = nz[k];
            }
#pragma unroll
            for (int k = 0; k < PW; ++k) zb[k] = nz[k];
            __syncthreads();
        }
    }
    float* out = partial + (int64_t)blockIdx.x * g.n_params;
    for (int i = t; i < g.n_params; i += PBT) out[i] = gacc[i];
}

__global__ void reduce_params(const float* __restrict__ partial, int n_cta, int64_t n, float* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    double s = 0.0;
    for (int c = 0; c < n_cta; ++c) s += partial[(int64_t)c * n + i];
    out[i] = (float)s;
}

inline unsigned g1(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

geraf_status proposal_saved_bytes(const geraf_proposal* p, size_t* bytes) {
    PropGeom g;
    if (!make_prop(p, &g)) return GERAF_ERR_INVALID_ARG;
    *bytes = (size_t)g.NH * g.W * g.n_cells * sizeof(float);
    return GERAF_OK;
}

geraf_status proposal_density_impl(const geraf_proposal* p, float* logits, float* q, void* saved, size_t saved_bytes,
                                   cudaStream_t st) {
    PropGeom g;
    if (!make_prop(p, &g)) return GERAF_ERR_INVALID_ARG;
    if (saved && saved_bytes < (size_t)g.NH * g.W * g.n_cells * sizeof(float))
        return fail(GERAF_ERR_WORKSPACE, "proposal_density: saved buffer too small");
    {
        const geraf_status as = smem_attrs((int)prop_forward_smem(g), "shared-memory opt-in", prop_forward_kernel);
        if (as != GERAF_OK) return as;
    }
    prop_forward_kernel<<<g1(g.n_cells, PFT), PFT, prop_forward_smem(g), st>>>(
        g, static_cast<const __half*>(p->features), p->params, logits, static_cast<float*>(saved));
    if (q) prop_q_kernel<<<g1((int64_t)g.G0 * g.G1, 128), 128, 0, st>>>(g, logits, q);
    return cuda_status(cudaGetLastError(), "proposal_density");
}

geraf_status sample_proposal_impl(const geraf_grid* gr, const geraf_proposal* p, const float* q, uint64_t seed,
                                  uint64_t step, float* xyz, float* apr, int32_t* idx, cudaStream_t st) {
    PropGeom g;
    if (!make_prop(p, &g)) return GERAF_ERR_INVALID_ARG;
    const float pz_cell = (float)((double)gr->pitch[2] * (double)gr->n[2] / (double)g.G2);
    const int64_t n_ray = (int64_t)gr->n[0] * gr->n[1];
    prop_sample_kernel<<<g1(n_ray, 128), 128, 0, st>>>(*gr, g, q, seed, step, pz_cell, xyz, apr, idx);
    return cuda_status(cudaGetLastError(), "sample_proposal");
}

geraf_status sample_cells_impl(const geraf_grid* gr, const geraf_proposal* p, const float* q, int32_t m,
                               int32_t r_max, int32_t dilate, uint64_t seed, uint64_t step, float* xyz, float* apr,
                               int32_t* idx, float* keep, void* ws, size_t* ws_bytes, cudaStream_t st) {
    PropGeom g;
    if (!make_prop(p, &g)) return GERAF_ERR_INVALID_ARG;
    if (gr->n[2] % g.G2 != 0 || gr->n[0] % g.G0 != 0 || gr->n[1] % g.G1 != 0)
        return fail(GERAF_ERR_INVALID_ARG, "sample_cells: the grid's columns and depths must be multiples of the "
                                           "proposal grid's");
    if (m < 1 || m > g.G2 || r_max < 0 || r_max > m || dilate < 0 || dilate >= g.G2)
        return fail(GERAF_ERR_INVALID_ARG, "sample_cells: need 1 <= m <= G2, 0 <= r_max <= m, 0 <= dilate < G2");
    const int s_fine = gr->n[2] / g.G2;
    const int n_out = m * s_fine + r_max;
    const int plane = g.G0 * g.G1;
    WsCarver c(ws);
    int32_t* table = c.take<int32_t>((size_t)plane * n_out);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used) return fail(GERAF_ERR_WORKSPACE, "sample_cells: workspace %zu < %zu bytes", *ws_bytes, c.used);
    cells_select_kernel<<<plane, 256, 0, st>>>(g, s_fine, m, r_max, dilate, n_out, q, table);
    const int64_t n_ray = (int64_t)gr->n[0] * gr->n[1];
    cells_sample_kernel<<<g1(n_ray * n_out, 256), 256, 0, st>>>(*gr, g, s_fine, n_out, table, seed, step, xyz, apr,
                                                               idx, keep);
    return cuda_status(cudaGetLastError(), "sample_cells");
}

geraf_status sample_backward_impl(const geraf_proposal* p, const geraf_grid* gr, int32_t n_z, const float* alpha,
                                  const float* T, const int32_t* idx, const float* logits, const void* saved,
                                  float* d_params, float* d_features, double* loss, void* ws, size_t* ws_bytes,
                                  cudaStream_t st) {
    PropGeom g;
    if (!make_prop(p, &g)) return GERAF_ERR_INVALID_ARG;
    const int plane = g.G0 * g.G1;
    int n_cta = device_sm_count();
    const int64_t n_tiles = (g.n_cells + PBT - 1) / PBT;
    if (n_cta > n_tiles) n_cta = (int)n_tiles;
    WsCarver c(ws);
    double* hist = c.take<double>(g.n_cells);
    float* dlog = c.take<float>(g.n_cells);
    double* col_loss = c.take<double>(plane);
    float* partial = c.take<float>((size_t)n_cta * g.n_params);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used)
        return fail(GERAF_ERR_WORKSPACE, "sample_backward: workspace %zu < %zu bytes", *ws_bytes, c.used);
    if (idx) {
        int hb = 32;
        while (hb > 1 && (size_t)g.G2 * hb * sizeof(double) > 32768) hb /= 2;
        prop_hist_cols_kernel<<<g1(plane, hb), hb, (size_t)g.G2 * hb * sizeof(double), st>>>(*gr, g, n_z, alpha, T,
                                                                                            idx, hist);
    } else {
        prop_hist_kernel<<<g1(g.n_cells, 128), 128, 0, st>>>(*gr, g, n_z, alpha, T, idx, hist);
    }
    prop_loss_kernel<<<g1(plane, 128), 128, 0, st>>>(g, logits, hist, dlog, col_loss);
    if (loss) sum_doubles_1<<<1, 256, 0, st>>>(col_loss, plane, loss);
    const size_t smem = (size_t)(2 * g.n_params + 2 * PBT * PWS + PBT) * sizeof(float);
    {
        const geraf_status as = smem_attrs(220 * 1024, "shared-memory opt-in", prop_backward_kernel);
        if (as != GERAF_OK) return as;
    }
    prop_backward_kernel<<<n_cta, PBT, smem, st>>>(g, static_cast<const __half*>(p->features), p->params,
                                                   static_cast<const float*>(saved), dlog, d_features, partial);
    reduce_params<<<g1(g.n_params, 256), 256, 0, st>>>(partial, n_cta, g.n_params, d_params);
    return cuda_status(cudaGetLastError(), "sample_backward");
}

}  // namespace geraf
