// SDF + reflectiveness MLP (section 5.2; App. C): sinusoidal positional
// encoding (section 9.3) of the cube-normalised position, softplus(beta)
// hidden layers of width 128, head [f, a_logit], a = sigmoid(a_logit), and the
// SDF gradient G = grad f (the surface normal direction) by three forward-mode
// tangents carried through every layer. FP32 CUDA-core path.
//
// Forward: persistent CTAs of 256 threads; a tile is 32 points x 4 streams
// (value, d/dx, d/dy, d/dz) = 128 columns. Each layer is a 128 x K x 128 GEMM
// from shared memory with an 8 x 8 register tile per thread, followed by the
// fused epilogue (bias, softplus on the value, sigmoid(beta h) times the
// tangents). Pre-activations of every layer are saved for the adjoint.
// Adjoint: one kernel for the head, one per hidden layer (top down). Each
// computes the pre-activation adjoint tile, accumulates the layer's weight
// gradient in registers across the CTA's tiles (a GEMM reducing over the
// 128 columns) and propagates the activation adjoint (a GEMM with W^T) in
// place. Per-CTA weight-gradient partials are summed in FP64 in a fixed order.
#include <math.h>

#include "common.cuh"

namespace geraf {

namespace {

constexpr int MW = 128;        // hidden width
constexpr int MTP = 32;        // points per tile
constexpr int MCOL = 4 * MTP;  // columns per tile
constexpr int XS = 132;        // padded shared-memory row stride (floats)
constexpr int MTHREADS = 256;

struct MlpGeom {
    int L, K0, NH;
    float beta, cx, cy, cz, half;
    int64_t n;
    int n_tiles;
    int64_t n_params;
    int64_t off_w[8], off_b[8];   // per layer (hidden layers then head)
    int k_in[8];
    float wk[21];                 // 2^k pi / half: x-derivative factor of octave k
};

bool make_geom(const geraf_field_desc* d, int64_t n, MlpGeom* g) {
    if (d->width != MW) {
        set_error("fields: MLP width %d unsupported (128 only)", d->width);
        return false;
    }
    if (d->n_levels < 1 || 6 * d->n_levels > MW || d->n_hidden < 1 || d->n_hidden > 7 || !(d->half > 0.0f)) {
        set_error("fields: MLP needs 1 <= n_levels <= 21, 1 <= n_hidden <= 7, half > 0");
        return false;
    }
    g->L = d->n_levels;
    g->K0 = 6 * d->n_levels;
    g->NH = d->n_hidden;
    g->beta = d->beta;
    g->cx = d->center[0]; g->cy = d->center[1]; g->cz = d->center[2];
    g->half = d->half;
    g->n = n;
    g->n_tiles = (int)((n + MTP - 1) / MTP);
    int64_t off = 0;
    for (int l = 0; l <= g->NH; ++l) {
        const int kin = l == 0 ? g->K0 : MW;
        const int out = l == g->NH ? 2 : MW;
        g->k_in[l] = kin;
        g->off_w[l] = off; off += (int64_t)out * kin;
        g->off_b[l] = off; off += out;
    }
    g->n_params = off;
    for (int k = 0; k < g->L; ++k) g->wk[k] = (float)((double)(1 << k) * 3.14159265358979323846 / (double)g->half);
    return true;
}

__device__ __forceinline__ float softplus_b(float h, float beta) {
    return fmaxf(h, 0.0f) + log1pf(expf(-beta * fabsf(h))) / beta;
}
__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + expf(-x)); }

// Positional encoding of tile points j0 .. j0+31 with their x-derivatives.
// Column c = 4 p + s (s = 0 value, 1..3 d/dx_{s-1}); feature k in 0 .. K0-1.
// T = false: X[k * XS + c]; T = true: X[c * XS + k].
template <bool T>
__device__ void pe_tile(float* X, const float* __restrict__ xyz, const MlpGeom& g, int64_t j0) {
    const int t = threadIdx.x;
    if (t >= 3 * MTP) return;
    const int p = t / 3, d = t - 3 * (t / 3);
    int64_t j = j0 + p;
    if (j >= g.n) j = g.n - 1;
    const float x = xyz[d * g.n + j];
    const float c = d == 0 ? g.cx : (d == 1 ? g.cy : g.cz);
    const double xt = ((double)x - (double)c) / (double)g.half;
    for (int k = 0; k < g.L; ++k) {
        const double t2 = xt * (double)(1 << k);
        const double r = t2 - 2.0 * rint(0.5 * t2);          // exact reduction mod 2
        float sn, cs;
        sincospif((float)r, &sn, &cs);                        // sin, cos of 2^k pi xt
        const float wk = g.wk[k];
        const int fs = 6 * k + d, fc = 6 * k + 3 + d;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float vs, vc;
            if (s == 0) { vs = sn; vc = cs; }
            else if (s - 1 == d) { vs = wk * cs; vc = -wk * sn; }
            else { vs = 0.0f; vc = 0.0f; }
            const int col = 4 * p + s;
            if (T) { X[col * XS + fs] = vs; X[col * XS + fc] = vc; }
            else { X[fs * XS + col] = vs; X[fc * XS + col] = vc; }
        }
    }
}

struct FwdArgs {
    MlpGeom g;
    const float* params;
    const float* xyz;
    float* sdf;
    float* grad;
    float* refl;
    float* saved;   // [NH][n][4][128] pre-activations, then [n] reflectiveness; may be null
};

// RU = output units per thread (8 x RU register tile): 8 gives 256 threads,
// 4 gives 512 threads (twice the warps per SM for the same shared tiles)
#ifndef GERAF_MLP_FWD_RU
#define GERAF_MLP_FWD_RU 4
#endif
constexpr int FRU = GERAF_MLP_FWD_RU;
constexpr int FT = 16 * (MW / FRU);

__global__ void __launch_bounds__(FT, 1) mlp_fwd_kernel(const FwdArgs a) {
    extern __shared__ __align__(16) float sm[];
    float* X0 = sm;
    float* X1 = X0 + MW * XS;
    float* Wt = X1 + MW * XS;             // W[u][k], rows padded to XS
    float* bias = Wt + MW * XS;           // [128]
    float* head = bias + MW;              // [2][128], then 2 biases
    const MlpGeom& g = a.g;
    const int t = threadIdx.x;
    const int ub = t >> 4, cb = t & 15;

    for (int i = t; i < 2 * MW; i += FT) head[i] = a.params[g.off_w[g.NH] + i];
    if (t < 2) head[2 * MW + t] = a.params[g.off_b[g.NH] + t];
    for (int i = t; i < MW * XS; i += FT) X0[i] = 0.0f;
    __syncthreads();

    for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x) {
        const int64_t j0 = (int64_t)tile * MTP;
        pe_tile<false>(X0, a.xyz, g, j0);
        float* Xin = X0;
        float* Xout = X1;
        for (int l = 0; l < g.NH; ++l) {
            const int K = g.k_in[l];
            const int Kp = (K + 3) & ~3;                 // K rounded up to the float4 step
            const float* W = a.params + g.off_w[l];
            // W [u][k] into shared memory as it lies in memory (rows padded to
            // XS, columns K .. Kp-1 zero): asynchronous 16-byte copies when the
            // rows are 16-byte aligned
            if ((K & 3) == 0 && (reinterpret_cast<uintptr_t>(W) & 15) == 0) {
                for (int idx = t; idx < MW * (K / 4); idx += FT) {
                    const int u = idx / (K / 4), kq = idx - u * (K / 4);
                    cp_async16(Wt + u * XS + 4 * kq, W + (int64_t)u * K + 4 * kq, 16);
                }
                cp_async_wait_all();
            } else {
                for (int idx = t; idx < MW * Kp; idx += FT) {
                    const int u = idx / Kp, k = idx - u * Kp;
                    Wt[u * XS + k] = k < K ? W[(int64_t)u * K + k] : 0.0f;
                }
            }
            if (t < MW) bias[t] = a.params[g.off_b[l] + t];
            __syncthreads();
            float acc[FRU][8];
#pragma unroll
            for (int i = 0; i < FRU; ++i)
#pragma unroll
                for (int jj = 0; jj < 8; ++jj) acc[i][jj] = 0.0f;
            for (int kq = 0; kq < Kp / 4; ++kq) {
                float4 wq[FRU];
#pragma unroll
                for (int i = 0; i < FRU; ++i)
                    wq[i] = *reinterpret_cast<const float4*>(Wt + (FRU * ub + i) * XS + 4 * kq);
#pragma unroll
                for (int m = 0; m < 4; ++m) {
                    const int k = 4 * kq + m;
                    const float4 x0 = *reinterpret_cast<const float4*>(Xin + k * XS + 4 * cb);
                    const float4 x1 = *reinterpret_cast<const float4*>(Xin + k * XS + 64 + 4 * cb);
                    const float xv[8] = {x0.x, x0.y, x0.z, x0.w, x1.x, x1.y, x1.z, x1.w};
#pragma unroll
                    for (int i = 0; i < FRU; ++i) {
                        const float wv = m == 0 ? wq[i].x : (m == 1 ? wq[i].y : (m == 2 ? wq[i].z : wq[i].w));
#pragma unroll
                        for (int jj = 0; jj < 8; ++jj) acc[i][jj] = fmaf(wv, xv[jj], acc[i][jj]);
                    }
                }
            }
            // epilogue: value column (bias, softplus) and tangents (sigmoid(beta h) * dh)
#pragma unroll
            for (int i = 0; i < FRU; ++i) {
                const int u = FRU * ub + i;
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int col0 = pp * 64 + 4 * cb;
                    const float h = acc[i][4 * pp] + bias[u];
                    const float sg = sigm(g.beta * h);
                    *reinterpret_cast<float4*>(Xout + u * XS + col0) =
                        make_float4(softplus_b(h, g.beta), sg * acc[i][4 * pp + 1], sg * acc[i][4 * pp + 2],
                                    sg * acc[i][4 * pp + 3]);
                    acc[i][4 * pp] = h;
                }
            }
            if (a.saved) {
#pragma unroll
                for (int pp = 0; pp < 2; ++pp) {
                    const int64_t j = j0 + pp * 16 + cb;
                    if (j < g.n) {
#pragma unroll
                        for (int s = 0; s < 4; ++s) {
                            float* dst = a.saved + (((int64_t)l * g.n + j) * 4 + s) * MW + FRU * ub;
#pragma unroll
                            for (int q = 0; q < FRU; q += 4)
                                *reinterpret_cast<float4*>(dst + q) = make_float4(
                                    acc[q][4 * pp + s], acc[q + 1][4 * pp + s], acc[q + 2][4 * pp + s],
                                    acc[q + 3][4 * pp + s]);
                        }
                    }
                }
            }
            __syncthreads();
            float* tmp = Xin; Xin = Xout; Xout = tmp;
        }
        // head: f and a_logit on value columns, G on tangent columns
        if (t < MCOL) {
            const int c = t, p = c >> 2, s = c & 3;
            const int64_t j = j0 + p;
            float v0 = 0.0f, v1 = 0.0f;
            for (int u = 0; u < MW; ++u) {
                const float x = Xin[u * XS + c];
                v0 = fmaf(head[u], x, v0);
                v1 = fmaf(head[MW + u], x, v1);
            }
            if (j < g.n) {
                if (s == 0) {
                    a.sdf[j] = v0 + head[2 * MW];
                    const float av = sigm(v1 + head[2 * MW + 1]);
                    if (a.refl) a.refl[j] = av;
                    if (a.saved) a.saved[(int64_t)g.NH * g.n * 4 * MW + j] = av;
                } else if (a.grad) {
                    a.grad[(int64_t)(s - 1) * g.n + j] = v0;
                }
            }
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------- adjoint
struct BwdArgs {
    MlpGeom g;
    const float* params;
    const float* xyz;
    const float* saved;
    const float* d_sdf;
    const float* d_grad;
    const float* d_refl;
    float* zbar;        // [n][4][128] activation adjoint, updated in place layer by layer
    float* partial;     // [gridDim.x][n_params]
    int layer;          // hidden layer index for the layer kernel
};

// head: dL/dW_head, dL/db_head and the adjoint of the last hidden activation.
// HT threads = HG groups of 128 (one unit each); group q takes points
// base + HG r + q; the groups' sums are added in a fixed order.
constexpr int HT = 1024;
constexpr int HG = HT / MW;
__global__ void __launch_bounds__(HT) mlp_head_bwd_kernel(const BwdArgs a) {
    __shared__ float red[2][HT];
    __shared__ float redb[2][HG];
    const MlpGeom& g = a.g;
    const int t = threadIdx.x, u = t & (MW - 1), grp = t >> 7;
    const float* Wh = a.params + g.off_w[g.NH];
    const float w0 = Wh[u], w1 = Wh[MW + u];
    const float* hsv = a.saved + (int64_t)(g.NH - 1) * g.n * 4 * MW;
    const float* asv = a.saved + (int64_t)g.NH * g.n * 4 * MW;
    float gw0 = 0.0f, gw1 = 0.0f, gb0 = 0.0f, gb1 = 0.0f;
    constexpr int R = 4;                                   // points per thread per round, loads in flight
    for (int64_t base = (int64_t)blockIdx.x * HG * R; base < g.n; base += (int64_t)gridDim.x * HG * R) {
        float df[R], dl[R], dG[R][3], h0[R], hd[R][3];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t j = base + HG * r + grp;
            const bool ok = j < g.n;
            const int64_t jj = ok ? j : 0;
            const float* h = hsv + jj * 4 * MW;
            df[r] = ok && a.d_sdf ? a.d_sdf[jj] : 0.0f;
            const float av = asv[jj];
            dl[r] = ok && a.d_refl ? a.d_refl[jj] * av * (1.0f - av) : 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                dG[r][d] = ok && a.d_grad ? a.d_grad[(int64_t)d * g.n + jj] : 0.0f;
                hd[r][d] = h[(d + 1) * MW + u];
            }
            h0[r] = h[u];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t j = base + HG * r + grp;
            if (j >= g.n) continue;
            const float sg = sigm(g.beta * h0[r]);
            const float z = softplus_b(h0[r], g.beta);
            gw0 += df[r] * z;
            gw1 += dl[r] * z;
            float* zb = a.zbar + j * 4 * MW;
            zb[u] = w0 * df[r] + w1 * dl[r];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                gw0 += dG[r][d] * sg * hd[r][d];
                zb[(d + 1) * MW + u] = w0 * dG[r][d];
            }
            if (u == 0) { gb0 += df[r]; gb1 += dl[r]; }
        }
    }
    red[0][t] = gw0;
    red[1][t] = gw1;
    if (u == 0) { redb[0][grp] = gb0; redb[1][grp] = gb1; }
    __syncthreads();
    float* out = a.partial + (int64_t)blockIdx.x * g.n_params;
    if (t < MW) {
        float s0 = 0.0f, s1 = 0.0f;
        for (int q = 0; q < HG; ++q) {
            s0 += red[0][q * MW + t];
            s1 += red[1][q * MW + t];
        }
        out[g.off_w[g.NH] + t] = s0;
        out[g.off_w[g.NH] + MW + t] = s1;
    }
    if (t == 0) {
        float b0 = 0.0f, b1 = 0.0f;
        for (int q = 0; q < HG; ++q) {
            b0 += redb[0][q];
            b1 += redb[1][q];
        }
        out[g.off_b[g.NH]] = b0;
        out[g.off_b[g.NH] + 1] = b1;
    }
}

// Rows c = 4 p + s of a [n][4][128] array for the tile's points j0 + p into a
// [128][XS] shared tile, all in flight at once; rows of points >= n read as 0.
__device__ __forceinline__ void stage_rows(float* dst, const float* src, int64_t j0, int64_t n) {
    for (int i = threadIdx.x; i < MCOL * (MW / 4); i += blockDim.x) {
        const int c = i >> 5, q = i & 31;
        const bool ok = j0 + (c >> 2) < n;
        cp_async16(dst + c * XS + 4 * q, ok ? src + (j0 * 4 + c) * MW + 4 * q : src, ok ? 16 : 0);
    }
}

// BU = rows of each thread's register tiles: 8 gives 256 threads, 4 gives 512
// threads (twice the warps per SM for the same shared tiles)
#ifndef GERAF_MLP_BWD_BU
#define GERAF_MLP_BWD_BU 8
#endif
constexpr int BU = GERAF_MLP_BWD_BU;
constexpr int BT = 16 * (MW / BU);

// hidden layer `layer`: pre-activation adjoint, weight/bias gradient, adjoint of the layer input
__global__ void __launch_bounds__(BT, 1) mlp_layer_bwd_kernel(const BwdArgs a) {
    extern __shared__ __align__(16) float sm[];
    float* HbT = sm;                 // [128 c][XS]  HbT[c][u]
    float* ZT = HbT + MCOL * XS;     // [128 c][XS]  ZT[c][k]
    float* Ws = ZT + MCOL * XS;      // [128 u][XS]  W[u][k]
    float* redb = Ws + MW * XS;      // [BT]
    const MlpGeom& g = a.g;
    const int li = a.layer;
    const int K = g.k_in[li];
    const int t = threadIdx.x;
    const float* W = a.params + g.off_w[li];
    for (int idx = t; idx < MW * K; idx += BT) {
        const int u = idx / K, k = idx - u * K;
        Ws[u * XS + k] = W[idx];
    }
    for (int i = t; i < MCOL * XS; i += BT) ZT[i] = 0.0f;
    __syncthreads();

    constexpr int EG = BT / MW;                  // elementwise groups
    const int ub = t >> 4, kb = t & 15;          // weight-gradient tile: units BU ub + i, inputs 4 kb (+64)
    const int kq = t >> 4, cq = t & 15;          // input-adjoint tile: inputs BU kq + kk, columns cq + 16 i
    const int eu = t & (MW - 1), eg = t >> 7;    // elementwise mapping
    float accw[BU][8];
#pragma unroll
    for (int i = 0; i < BU; ++i)
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) accw[i][jj] = 0.0f;
    float accb = 0.0f;
    const float* hs = a.saved + (int64_t)li * g.n * 4 * MW;
    const float* hin = li > 0 ? a.saved + (int64_t)(li - 1) * g.n * 4 * MW : nullptr;

    for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x) {
        const int64_t j0 = (int64_t)tile * MTP;
        // pre-activation adjoint (HbT), computed in place from the staged
        // activation adjoint (in HbT) and pre-activations (in ZT)
        stage_rows(HbT, a.zbar, j0, g.n);
        stage_rows(ZT, hs, j0, g.n);
        cp_async_wait_all();
        __syncthreads();
#pragma unroll 4
        for (int p = eg; p < MTP; p += EG) {
            float* hb = HbT + 4 * p * XS + eu;
            const float* h = ZT + 4 * p * XS + eu;
            const float h0 = h[0];
            const float sg = sigm(g.beta * h0);
            const float dsg = g.beta * sg * (1.0f - sg);
            const float z0 = hb[0], z1 = hb[XS], z2 = hb[2 * XS], z3 = hb[3 * XS];
            const float b0 = z0 * sg + (z1 * h[XS] + z2 * h[2 * XS] + z3 * h[3 * XS]) * dsg;
            accb += b0;                                   // 0 for points >= n (staged zeros)
            hb[0] = b0;
            hb[XS] = sg * z1;
            hb[2 * XS] = sg * z2;
            hb[3 * XS] = sg * z3;
        }
        __syncthreads();
        // input activations (ZT) of the layer: from the previous layer's pre-activations
        if (hin) {
            stage_rows(ZT, hin, j0, g.n);
            cp_async_wait_all();
            __syncthreads();
#pragma unroll 4
            for (int p = eg; p < MTP; p += EG) {
                float* z = ZT + 4 * p * XS + eu;
                const float x0 = z[0];
                const float s0 = sigm(g.beta * x0);
                z[0] = softplus_b(x0, g.beta);
                z[XS] *= s0;
                z[2 * XS] *= s0;
                z[3 * XS] *= s0;
            }
        }
        // first layer: its input is the positional encoding (columns of points beyond n
        // meet a zero HbT and contribute nothing)
        if (!hin) pe_tile<true>(ZT, a.xyz, g, j0);
        // the next tile's rows (contiguous 2 KB per point in each array) head for
        // L2 while this tile's two products run, so its staging reads L2
        const int next = tile + gridDim.x;
        if (t == 0 && next < g.n_tiles) {
            const int64_t jn = (int64_t)next * MTP;
            const uint32_t bytes = (uint32_t)(min((int64_t)MTP, g.n - jn) * 4 * MW * sizeof(float));
            prefetch_l2_bulk(a.zbar + jn * 4 * MW, bytes);
            prefetch_l2_bulk(hs + jn * 4 * MW, bytes);
            if (hin) prefetch_l2_bulk(hin + jn * 4 * MW, bytes);
        }
        __syncthreads();
        // weight gradient: accw[u][k] += sum_c HbT[c][u] ZT[c][k]; an input width of
        // at most 64 (the encoding layer) leaves the upper half of the k tile zero
        if (K > 64) {
#pragma unroll 2
            for (int c = 0; c < MCOL; ++c) {
                float hv[BU];
#pragma unroll
                for (int q = 0; q < BU; q += 4) {
                    const float4 h4 = *reinterpret_cast<const float4*>(HbT + c * XS + BU * ub + q);
                    hv[q] = h4.x; hv[q + 1] = h4.y; hv[q + 2] = h4.z; hv[q + 3] = h4.w;
                }
                const float4 z0 = *reinterpret_cast<const float4*>(ZT + c * XS + 4 * kb);
                const float4 z1 = *reinterpret_cast<const float4*>(ZT + c * XS + 64 + 4 * kb);
                const float zv[8] = {z0.x, z0.y, z0.z, z0.w, z1.x, z1.y, z1.z, z1.w};
#pragma unroll
                for (int i = 0; i < BU; ++i)
#pragma unroll
                    for (int jj = 0; jj < 8; ++jj) accw[i][jj] = fmaf(hv[i], zv[jj], accw[i][jj]);
            }
        } else if (4 * kb < K) {
#pragma unroll 2
            for (int c = 0; c < MCOL; ++c) {
                float hv[BU];
#pragma unroll
                for (int q = 0; q < BU; q += 4) {
                    const float4 h4 = *reinterpret_cast<const float4*>(HbT + c * XS + BU * ub + q);
                    hv[q] = h4.x; hv[q + 1] = h4.y; hv[q + 2] = h4.z; hv[q + 3] = h4.w;
                }
                const float4 z0 = *reinterpret_cast<const float4*>(ZT + c * XS + 4 * kb);
                const float zv[4] = {z0.x, z0.y, z0.z, z0.w};
#pragma unroll
                for (int i = 0; i < BU; ++i)
#pragma unroll
                    for (int jj = 0; jj < 4; ++jj) accw[i][jj] = fmaf(hv[i], zv[jj], accw[i][jj]);
            }
        }
        // adjoint of the layer input: zbar[c][k] = sum_u HbT[c][u] W[u][k]  (in place)
        if (hin) {
            float acc[8][BU];
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int kk = 0; kk < BU; ++kk) acc[i][kk] = 0.0f;
            for (int u = 0; u < MW; u += 4) {
                float4 hv[8];
#pragma unroll
                for (int i = 0; i < 8; ++i) hv[i] = *reinterpret_cast<const float4*>(HbT + (cq + 16 * i) * XS + u);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    float wv[BU];
#pragma unroll
                    for (int r = 0; r < BU; r += 4) {
                        const float4 w4 = *reinterpret_cast<const float4*>(Ws + (u + q) * XS + BU * kq + r);
                        wv[r] = w4.x; wv[r + 1] = w4.y; wv[r + 2] = w4.z; wv[r + 3] = w4.w;
                    }
#pragma unroll
                    for (int i = 0; i < 8; ++i) {
                        const float hq = q == 0 ? hv[i].x : (q == 1 ? hv[i].y : (q == 2 ? hv[i].z : hv[i].w));
#pragma unroll
                        for (int kk = 0; kk < BU; ++kk) acc[i][kk] = fmaf(hq, wv[kk], acc[i][kk]);
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = cq + 16 * i, p = c >> 2, s = c & 3;
                const int64_t j = j0 + p;
                if (j < g.n) {
                    float* dst = a.zbar + (j * 4 + s) * MW + BU * kq;
#pragma unroll
                    for (int r = 0; r < BU; r += 4)
                        *reinterpret_cast<float4*>(dst + r) =
                            make_float4(acc[i][r], acc[i][r + 1], acc[i][r + 2], acc[i][r + 3]);
                }
            }
        }
        __syncthreads();
    }
    // per-CTA partials
    float* out = a.partial + (int64_t)blockIdx.x * g.n_params;
#pragma unroll
    for (int i = 0; i < BU; ++i) {
        const int u = BU * ub + i;
#pragma unroll
        for (int jj = 0; jj < 8; ++jj) {
            const int k = jj < 4 ? 4 * kb + jj : 64 + 4 * kb + (jj - 4);
            if (k < K) out[g.off_w[li] + (int64_t)u * K + k] = accw[i][jj];
        }
    }
    redb[t] = accb;
    __syncthreads();
    if (t < MW) {
        float sb = 0.0f;
        for (int q = 0; q < EG; ++q) sb += redb[t + q * MW];
        out[g.off_b[li] + t] = sb;
    }
}

__global__ void reduce_partials(const float* __restrict__ partial, int n_cta, int64_t n_params,
                                float* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n_params) return;
    double s = 0.0;
    for (int c = 0; c < n_cta; ++c) s += partial[(int64_t)c * n_params + i];
    out[i] = (float)s;
}

size_t fwd_smem() { return (size_t)(3 * MW * XS + MW + 2 * MW + 2) * sizeof(float); }
size_t bwd_smem() { return (size_t)(2 * MCOL * XS + MW * XS + BT) * sizeof(float); }

int n_ctas_for(int n_tiles) {
    const int sms = device_sm_count();
    return n_tiles < sms ? (n_tiles > 0 ? n_tiles : 1) : sms;
}

}  // namespace

bool mlp_is_wide(const geraf_field_desc* d);
geraf_status mlp_wide_saved_bytes(const geraf_field_desc* d, int64_t n, size_t* bytes);
geraf_status mlp_wide_forward(const geraf_field_desc* d, const float* xyz, int64_t n, float* sdf, float* grad,
                              float* refl, void* saved, size_t saved_bytes, cudaStream_t st);
geraf_status mlp_wide_backward(const geraf_field_desc* d, const float* xyz, int64_t n, const void* saved,
                               const float* d_sdf, const float* d_grad, const float* d_refl, float* d_params,
                               void* ws, size_t* ws_bytes, cudaStream_t st);

geraf_status mlp_saved_bytes(const geraf_field_desc* d, int64_t n, size_t* bytes) {
    if (mlp_is_wide(d)) return mlp_wide_saved_bytes(d, n, bytes);
    MlpGeom g;
    if (!make_geom(d, n, &g)) return GERAF_ERR_UNSUPPORTED;
    *bytes = ((size_t)g.NH * n * 4 * MW + (size_t)n) * sizeof(float);
    return GERAF_OK;
}

geraf_status mlp_tc_forward_impl(const geraf_field_desc*, const float*, int64_t, float*, float*, float*, void*,
                                 cudaStream_t);

geraf_status mlp_forward_impl(const geraf_field_desc* d, const float* xyz, int64_t n, float* sdf, float* grad,
                              float* refl, void* saved, size_t saved_bytes, cudaStream_t st) {
    if (mlp_is_wide(d)) return mlp_wide_forward(d, xyz, n, sdf, grad, refl, saved, saved_bytes, st);
    MlpGeom g;
    if (!make_geom(d, n, &g)) return GERAF_ERR_UNSUPPORTED;
    if (d->precision != GERAF_PREC_FP32 && d->precision != GERAF_PREC_BF16)
        return fail(GERAF_ERR_UNSUPPORTED, "fields: MLP precision %d unknown", d->precision);
    if (saved) {
        size_t need = 0;
        mlp_saved_bytes(d, n, &need);
        if (saved_bytes < need) return fail(GERAF_ERR_WORKSPACE, "fields: saved %zu < %zu bytes", saved_bytes, need);
    }
    if (d->precision == GERAF_PREC_BF16) return mlp_tc_forward_impl(d, xyz, n, sdf, grad, refl, saved, st);
    {
        const geraf_status as = smem_attrs((int)fwd_smem(), "shared-memory opt-in", mlp_fwd_kernel);
        if (as != GERAF_OK) return as;
    }
    FwdArgs a{g, d->params, xyz, sdf, grad, refl, static_cast<float*>(saved)};
    mlp_fwd_kernel<<<n_ctas_for(g.n_tiles), FT, fwd_smem(), st>>>(a);
    return cuda_status(cudaGetLastError(), "fields(mlp)");
}

int mlp_tc_backward_ctas(int64_t n);
geraf_status mlp_tc_backward_impl(const geraf_field_desc* d, const float* xyz, int64_t n, const void* saved,
                                  const float* d_sdf, const float* d_grad, const float* d_refl, float* zbar,
                                  float* partial, int64_t n_params, int n_cta, cudaStream_t st);

geraf_status mlp_backward_impl(const geraf_field_desc* d, const float* xyz, int64_t n, const void* saved,
                               const float* d_sdf, const float* d_grad, const float* d_refl, float* d_params,
                               void* ws, size_t* ws_bytes, cudaStream_t st) {
    if (mlp_is_wide(d))
        return mlp_wide_backward(d, xyz, n, saved, d_sdf, d_grad, d_refl, d_params, ws, ws_bytes, st);
    MlpGeom g;
    if (!make_geom(d, n, &g)) return GERAF_ERR_UNSUPPORTED;
    // BF16 networks: the straight-through adjoint on tcgen05 tensor cores; FP32
    // networks: CUDA cores. Both leave per-CTA partials reduced here in FP64.
    const bool bf16 = d->precision == GERAF_PREC_BF16;
    const int n_cta = bf16 ? mlp_tc_backward_ctas(n) : n_ctas_for(g.n_tiles);
    WsCarver c(ws);
    float* zbar = c.take<float>((size_t)n * 4 * MW);
    float* partial = c.take<float>((size_t)n_cta * g.n_params);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used)
        return fail(GERAF_ERR_WORKSPACE, "fields_backward: workspace %zu < %zu bytes", *ws_bytes, c.used);
    if (bf16) {
        geraf_status s = mlp_tc_backward_impl(d, xyz, n, saved, d_sdf, d_grad, d_refl, zbar, partial, g.n_params,
                                              n_cta, st);
        if (s != GERAF_OK) return s;
        reduce_partials<<<(unsigned)((g.n_params + 255) / 256), 256, 0, st>>>(partial, n_cta, g.n_params, d_params);
        return cuda_status(cudaGetLastError(), "fields_backward(mlp bf16)");
    }
    {
        const geraf_status as = smem_attrs((int)bwd_smem(), "shared-memory opt-in", mlp_layer_bwd_kernel);
        if (as != GERAF_OK) return as;
    }
    BwdArgs a{g, d->params, xyz, static_cast<const float*>(saved), d_sdf, d_grad, d_refl, zbar, partial, 0};
    mlp_head_bwd_kernel<<<n_cta, HT, 0, st>>>(a);
    for (int l = g.NH - 1; l >= 0; --l) {
        a.layer = l;
        mlp_layer_bwd_kernel<<<n_cta, BT, bwd_smem(), st>>>(a);
    }
    reduce_partials<<<(unsigned)((g.n_params + 255) / 256), 256, 0, st>>>(partial, n_cta, g.n_params, d_params);
    return cuda_status(cudaGetLastError(), "fields_backward(mlp)");
}

}  // namespace geraf
