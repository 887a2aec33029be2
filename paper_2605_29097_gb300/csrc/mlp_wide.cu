// Field networks of any width and depth, in particular the paper's two
// networks (App. C "Training Setup": an SDF network of 8 softplus layers of
// 256 on a 10-octave positional encoding, and a separate reflectivity network
// of 4 layers of 256 on the same encoding; section 5.2 "Signal
// representation"), FP32 on CUDA cores (the BF16 form of these networks runs
// on the tensor cores: mlp_wide_tc.cu).
//
// Layer-major: the positional encoding, every layer and the head are separate
// launches over all points, with the pre-activations of each layer kept in the
// caller's `saved` buffer (they are the adjoint's inputs anyway). A layer is a
// GEMM over rows r = j S + s (point j, stream s: value and, for the SDF
// network, the three x-tangents, S = 4) with a 128 x 128 output tile per CTA,
// contraction chunks of 32 staged in shared memory (register prefetch of the
// next chunk under the current one's FMAs, two buffers) and an 8 x 8 register
// tile per thread. The activation z = softplus(h) (value row) and
// sigmoid(beta h0) dh (tangent rows) is applied while a chunk is staged, so no
// activation tensor is ever written. The adjoint runs the same GEMM core for
// the input adjoint (W^T) and for the weight gradient (a contraction over the
// rows of a split, partials summed in FP64 in a fixed order).
#include <math.h>

#include <algorithm>

#include "common.cuh"

namespace geraf {

namespace {

constexpr int GT = 256;          // threads per CTA
constexpr int GM = 128;          // output rows per tile
constexpr int GN = 128;          // output columns per tile
constexpr int GK = 32;           // contraction chunk
constexpr int GLD = GM + 4;      // shared row stride (floats)
constexpr int WMAX_LAYERS = 16;  // hidden layers of one network

struct WNet {
    const float* params;     // this network's packed parameters
    int L, K0, K0p;          // octaves, encoding width, encoding width padded to GK
    int W, NH, S, head_out;  // width, hidden layers, streams, head outputs
    float beta, cx, cy, cz, half;
    int64_t off_w[WMAX_LAYERS + 1], off_b[WMAX_LAYERS + 1];
    int64_t n_params;
    float wk[21];            // 2^k pi / half: x-derivative factor of octave k
    int k_in(int l) const { return l == 0 ? K0 : W; }
    int k_pad(int l) const { return l == 0 ? K0p : W; }
};

bool make_wnet(const float* params, int L, int W, int NH, int head_out, int S, const geraf_field_desc* d,
               WNet* g) {
    if (L < 1 || L > 21 || W < 32 || W > 1024 || (W % 32) != 0 || NH < 1 || NH > WMAX_LAYERS) {
        set_error("fields: wide MLP needs 1 <= n_levels <= 21, width a multiple of 32 in [32, 1024], "
                  "1 <= hidden layers <= %d", WMAX_LAYERS);
        return false;
    }
    if (!(d->half > 0.0f)) {
        set_error("fields: half > 0 required");
        return false;
    }
    g->params = params;
    g->L = L;
    g->K0 = 6 * L;
    g->K0p = (g->K0 + GK - 1) / GK * GK;
    g->W = W;
    g->NH = NH;
    g->S = S;
    g->head_out = head_out;
    g->beta = d->beta;
    g->cx = d->center[0]; g->cy = d->center[1]; g->cz = d->center[2];
    g->half = d->half;
    int64_t off = 0;
    for (int l = 0; l <= NH; ++l) {
        const int kin = l == 0 ? g->K0 : W;
        const int out = l == NH ? head_out : W;
        g->off_w[l] = off; off += (int64_t)out * kin;
        g->off_b[l] = off; off += out;
    }
    g->n_params = off;
    for (int k = 0; k < L; ++k) g->wk[k] = (float)((double)(1 << k) * 3.14159265358979323846 / (double)g->half);
    return true;
}

__device__ __forceinline__ float softplus_w(float h, float beta) {
    return fmaxf(h, 0.0f) + log1pf(expf(-beta * fabsf(h))) / beta;
}
__device__ __forceinline__ float sigm_w(float x) { return 1.0f / (1.0f + expf(-x)); }

// positional encoding rows of n points: Z0[(j S + s) K0p + f], zero beyond K0.
// Thread = (point, axis d); it owns every feature f with f % 3 == d.
__global__ void wpe_kernel(const float* __restrict__ xyz, int64_t n, WNet g, float* __restrict__ Z0) {
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (t >= 3 * n) return;
    const int64_t j = t / 3;
    const int d = (int)(t - 3 * j);
    const float x = xyz[d * n + j];
    const float c = d == 0 ? g.cx : (d == 1 ? g.cy : g.cz);
    const double xt = ((double)x - (double)c) / (double)g.half;
    for (int k = 0; k < g.L; ++k) {
        const double t2 = xt * (double)(1 << k);
        const double r = t2 - 2.0 * rint(0.5 * t2);          // exact reduction mod 2
        float sn, cs;
        sincospif((float)r, &sn, &cs);                        // sin, cos of 2^k pi xt
        const float wk = g.wk[k];
        const int fs = 6 * k + d, fc = 6 * k + 3 + d;
        for (int s = 0; s < g.S; ++s) {
            float vs, vc;
            if (s == 0) { vs = sn; vc = cs; }
            else if (s - 1 == d) { vs = wk * cs; vc = -wk * sn; }
            else { vs = 0.0f; vc = 0.0f; }
            float* row = Z0 + (j * g.S + s) * g.K0p;
            row[fs] = vs;
            row[fc] = vc;
        }
    }
    if (d == 0)
        for (int s = 0; s < g.S; ++s)
            for (int f = g.K0; f < g.K0p; ++f) Z0[(j * g.S + s) * g.K0p + f] = 0.0f;
}

// ------------------------------------------------------------------ GEMM core
enum { WG_FWD = 0, WG_DZ = 1, WG_DW = 2 };

struct WGemm {
    int64_t M;          // output rows
    int N;              // output columns
    int64_t Kc;         // contraction length (FWD, DZ: a multiple of GK)
    const float* a;     // FWD, DZ: [M][lda] along the contraction; DW: [rows][lda] (Hb, columns = units)
    int64_t lda;
    const float* b;     // FWD: W [N][ldb]; DZ: W [Kc][ldb]; DW: Z [rows][ldb]
    int64_t ldb;
    int act;            // FWD: activation of a; DW: activation of b
    int S;
    float beta;
    float* c;
    int64_t ldc;
    const float* bias;  // FWD: added on value rows
    int n_valid;        // DW: columns written (the layer's real input width)
    int64_t rows;       // DW: contraction rows in total
    int64_t rows_per_split;
    int64_t split_stride;   // DW: floats between the partial rows of two splits
};

// z of element (row r, column k) from pre-activations `h` (rows r, stride ld):
// softplus(h) on value rows, sigmoid(beta h0) h on tangent rows
__device__ __forceinline__ void act4(const float* __restrict__ h, int64_t ld, int64_t r, int64_t col, int S,
                                     float beta, float4& v) {
    const int s = (int)(r % S);
    if (s == 0) {
        v.x = softplus_w(v.x, beta); v.y = softplus_w(v.y, beta);
        v.z = softplus_w(v.z, beta); v.w = softplus_w(v.w, beta);
    } else {
        const float4 h0 = *reinterpret_cast<const float4*>(h + (r - s) * ld + col);
        v.x *= sigm_w(beta * h0.x); v.y *= sigm_w(beta * h0.y);
        v.z *= sigm_w(beta * h0.z); v.w *= sigm_w(beta * h0.w);
    }
}

// 16 floats src[off .. off+15]: one row segment of an activation buffer
// (16-byte aligned, `vec`) or of a weight matrix inside the packed parameters
// (any alignment; columns >= kvalid of the row read as 0)
template <bool VEC>
__device__ __forceinline__ void load16(const float* __restrict__ src, int64_t off, int64_t col, int64_t kvalid,
                                       float4 (&v)[4]) {
    if (VEC) {
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = *reinterpret_cast<const float4*>(src + off + 4 * q);
    } else {
        float t[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) t[e] = col + e < kvalid ? __ldg(src + off + e) : 0.0f;
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = make_float4(t[4 * q], t[4 * q + 1], t[4 * q + 2], t[4 * q + 3]);
    }
}

// Transposing staging: dst[kk][m] = src[(row0 + m) * ld + k0 + kk], rows >= nrows
// (and columns >= kvalid) read as 0. Thread t: row m = t / 2, 16 consecutive kk.
template <bool VEC>
struct LoadT {
    float4 v[4];
    __device__ __forceinline__ void fetch(const float* __restrict__ src, int64_t ld, int64_t row0, int64_t nrows,
                                          int64_t k0, int64_t kvalid, int act, int S, float beta) {
        const int m = threadIdx.x >> 1, kh = (threadIdx.x & 1) * 16;
        const int64_t r = row0 + m;
        if (r < nrows) {
            load16<VEC>(src, r * ld + k0 + kh, k0 + kh, kvalid, v);
            if (act)
#pragma unroll
                for (int q = 0; q < 4; ++q) act4(src, ld, r, k0 + kh + 4 * q, S, beta, v[q]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    __device__ __forceinline__ void store(float* dst) const {
        const int m = threadIdx.x >> 1, kh = (threadIdx.x & 1) * 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            dst[(kh + 4 * q + 0) * GLD + m] = v[q].x;
            dst[(kh + 4 * q + 1) * GLD + m] = v[q].y;
            dst[(kh + 4 * q + 2) * GLD + m] = v[q].z;
            dst[(kh + 4 * q + 3) * GLD + m] = v[q].w;
        }
    }
};

// Natural staging: dst[kk][c] = src[(k0 + kk) * ld + col0 + c], rows >= nk and
// columns >= ncols (a multiple of 16) read as 0. Thread t: kk = t / 8, 16 columns.
template <bool VEC>
struct LoadN {
    float4 v[4];
    __device__ __forceinline__ void fetch(const float* __restrict__ src, int64_t ld, int64_t k0, int64_t nk,
                                          int64_t col0, int64_t ncols, int act, int S, float beta) {
        const int kk = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 16;
        const int64_t r = k0 + kk;
        if (r < nk && col0 + c0 < ncols) {
            load16<VEC>(src, r * ld + col0 + c0, col0 + c0, ncols, v);
            if (act)
#pragma unroll
                for (int q = 0; q < 4; ++q) act4(src, ld, r, col0 + c0 + 4 * q, S, beta, v[q]);
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q) v[q] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
    }
    __device__ __forceinline__ void store(float* dst) const {
        const int kk = threadIdx.x >> 3, c0 = (threadIdx.x & 7) * 16;
#pragma unroll
        for (int q = 0; q < 4; ++q) *reinterpret_cast<float4*>(dst + kk * GLD + c0 + 4 * q) = v[q];
    }
};

template <int MODE>
#ifndef GERAF_WG_MINB
#define GERAF_WG_MINB 2
#endif
__global__ void __launch_bounds__(GT, GERAF_WG_MINB) wgemm_kernel(const WGemm p) {
    extern __shared__ __align__(16) float wsm[];
    float* As = wsm;                  // [2][GK][GLD]
    float* Bs = wsm + 2 * GK * GLD;   // [2][GK][GLD]
    const int t = threadIdx.x;
    const int ty = t >> 4, tx = t & 15;
    const int64_t m0 = (int64_t)blockIdx.y * GM;
    const int64_t n0 = (int64_t)blockIdx.x * GN;
    int64_t k_begin = 0, k_end = p.Kc;
    if (MODE == WG_DW) {
        k_begin = (int64_t)blockIdx.z * p.rows_per_split;
        k_end = min(p.rows, k_begin + p.rows_per_split);
    }
    const int64_t nch = k_end > k_begin ? (k_end - k_begin + GK - 1) / GK : 0;
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;

    // A operand staged as As[kk][m], B as Bs[kk][n]
    LoadT<true> lat;    // FWD, DZ: A is an activation buffer [M][contraction]
    LoadN<true> lan;    // DW: A (hbar) is [contraction rows][units]
    LoadT<false> lbt;   // FWD: B^T = W [N][contraction] (packed parameters)
    LoadN<false> lbw;   // DZ: W [contraction][N] (packed parameters)
    LoadN<true> lbz;    // DW: Z [contraction rows][N] (activation buffer)
    auto fetch = [&](int64_t kc) {
        if (MODE == WG_FWD) {
            lat.fetch(p.a, p.lda, m0, p.M, kc, p.lda, p.act, p.S, p.beta);
            lbt.fetch(p.b, p.ldb, n0, p.N, kc, p.ldb, 0, 1, 0.0f);
        } else if (MODE == WG_DZ) {
            lat.fetch(p.a, p.lda, m0, p.M, kc, p.lda, 0, 1, 0.0f);
            lbw.fetch(p.b, p.ldb, kc, p.Kc, n0, p.N, 0, 1, 0.0f);
        } else {
            lan.fetch(p.a, p.lda, kc, k_end, m0, p.M, 0, 1, 0.0f);
            lbz.fetch(p.b, p.ldb, kc, k_end, n0, p.ldb, p.act, p.S, p.beta);
        }
    };
    auto store = [&](int buf) {
        float* a = As + buf * GK * GLD;
        float* b = Bs + buf * GK * GLD;
        if (MODE == WG_FWD) { lat.store(a); lbt.store(b); }
        else if (MODE == WG_DZ) { lat.store(a); lbw.store(b); }
        else { lan.store(a); lbz.store(b); }
    };
    if (nch > 0) {
        fetch(k_begin);
        store(0);
    }
    __syncthreads();
    for (int64_t c = 0; c < nch; ++c) {
        const int buf = (int)(c & 1);
        if (c + 1 < nch) fetch(k_begin + (c + 1) * GK);
        const float* a = As + buf * GK * GLD;
        const float* b = Bs + buf * GK * GLD;
#pragma unroll 8
        for (int kk = 0; kk < GK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(a + kk * GLD + 4 * ty);
            const float4 a1 = *reinterpret_cast<const float4*>(a + kk * GLD + 64 + 4 * ty);
            const float4 b0 = *reinterpret_cast<const float4*>(b + kk * GLD + 4 * tx);
            const float4 b1 = *reinterpret_cast<const float4*>(b + kk * GLD + 64 + 4 * tx);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        if (c + 1 < nch) store(buf ^ 1);
        __syncthreads();
    }
    // epilogue: rows m0 + {4ty + i, 64 + 4ty + i}, columns n0 + {4tx + j, 64 + 4tx + j}
#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int64_t r = m0 + (i < 4 ? 4 * ty + i : 64 + 4 * ty + (i - 4));
        if (r >= p.M) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int64_t n = n0 + 64 * h + 4 * tx;
            float4 v = make_float4(acc[i][4 * h], acc[i][4 * h + 1], acc[i][4 * h + 2], acc[i][4 * h + 3]);
            if (MODE == WG_FWD) {
                if (n >= p.N) continue;
                if ((r % p.S) == 0) {
                    v.x += p.bias[n]; v.y += p.bias[n + 1]; v.z += p.bias[n + 2]; v.w += p.bias[n + 3];
                }
                *reinterpret_cast<float4*>(p.c + r * p.ldc + n) = v;
            } else if (MODE == WG_DZ) {
                if (n >= p.N) continue;
                *reinterpret_cast<float4*>(p.c + r * p.ldc + n) = v;
            } else {
                float* dst = p.c + (int64_t)blockIdx.z * p.split_stride + r * p.ldc;
                const float vv[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (n + q < p.n_valid) dst[n + q] = vv[q];
            }
        }
    }
}

size_t wgemm_smem() { return (size_t)4 * GK * GLD * sizeof(float); }

// ------------------------------------------------------------- head forward
// One warp per point: z of the last hidden layer, head rows, outputs.
// out_f / out_grad: row 0 is f (SDF network or shared trunk); a from row
// `a_row` (1 for the shared trunk, 0 for the reflectivity network, -1: none).
__global__ void whead_fwd_kernel(WNet g, int64_t n, const float* __restrict__ H, float* __restrict__ out_f,
                                 float* __restrict__ out_grad, float* __restrict__ out_a, float* __restrict__ a_saved,
                                 int a_row) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const float* Wh = g.params + g.off_w[g.NH];
    const float* bh = g.params + g.off_b[g.NH];
    const float* h0 = H + (j * g.S) * g.W;
    float acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};      // row0 x streams 0..3, a_row x value
    for (int u = lane; u < g.W; u += 32) {
        const float hv = h0[u];
        const float z0 = softplus_w(hv, g.beta);
        acc[0] = fmaf(Wh[u], z0, acc[0]);
        if (a_row > 0) acc[4] = fmaf(Wh[(int64_t)a_row * g.W + u], z0, acc[4]);
        if (g.S == 4 && out_grad) {
            const float sg = sigm_w(g.beta * hv);
#pragma unroll
            for (int s = 1; s < 4; ++s) acc[s] = fmaf(Wh[u], sg * h0[(int64_t)s * g.W + u], acc[s]);
        }
    }
#pragma unroll
    for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[q] += __shfl_xor_sync(0xffffffffu, acc[q], o);
    if (lane == 0) {
        if (out_f) out_f[j] = acc[0] + bh[0];
        if (out_grad && g.S == 4)
            for (int d = 0; d < 3; ++d) out_grad[(int64_t)d * n + j] = acc[1 + d];
        if (a_row >= 0) {
            const float a = sigm_w(a_row == 0 ? acc[0] + bh[0] : acc[4] + bh[a_row]);
            if (out_a) out_a[j] = a;
            if (a_saved) a_saved[j] = a;
        }
    }
}

// ------------------------------------------------------------- head adjoint
// Block (split, 32-unit chunk): threadIdx.x = unit u, threadIdx.y = one of 8
// point lanes over the split's points [sp*pps, ...). Writes the top activation
// adjoint zbar[(j S + s) W + u] and the head's gradient partials (lane sums
// added in a fixed order). For the reflectivity network (S = 1, head
// [a_logit]) the output adjoint is d_a a (1 - a); for the SDF network d_f with
// tangents d_grad; the shared trunk adds row 1 (a_logit).
__global__ void __launch_bounds__(256) whead_bwd_kernel(WNet g, int64_t n, int64_t pps, const float* __restrict__ H,
                                                        const float* __restrict__ a_saved,
                                                        const float* __restrict__ d_f,
                                                        const float* __restrict__ d_grad,
                                                        const float* __restrict__ d_a, int refl_net,
                                                        float* __restrict__ zbar, float* __restrict__ partial,
                                                        int64_t split_stride) {
    __shared__ float red[4][8][32];
    const int sp = blockIdx.x;
    const int u = blockIdx.y * 32 + threadIdx.x;
    const int64_t j0 = (int64_t)sp * pps, j1 = min(n, j0 + pps);
    const float* Wh = g.params + g.off_w[g.NH];
    float gw0 = 0.0f, gw1 = 0.0f, gb0 = 0.0f, gb1 = 0.0f;
    if (u < g.W) {
        const float w0 = Wh[u], w1 = g.head_out == 2 ? Wh[g.W + u] : 0.0f;
        for (int64_t j = j0 + threadIdx.y; j < j1; j += 8) {
            const float* h = H + (j * g.S) * g.W;
            const float hv = h[u];
            const float z0 = softplus_w(hv, g.beta);
            float dl = 0.0f;
            if (d_a && (refl_net || g.head_out == 2)) {
                const float a = a_saved[j];
                dl = d_a[j] * a * (1.0f - a);
            }
            const float df = refl_net ? dl : (d_f ? d_f[j] : 0.0f);
            float* zb = zbar + (j * g.S) * g.W;
            zb[u] = w0 * df + (refl_net ? 0.0f : w1 * dl);
            gw0 = fmaf(df, z0, gw0);
            if (!refl_net && g.head_out == 2) gw1 = fmaf(dl, z0, gw1);
            if (g.S == 4) {
                const float sg = sigm_w(g.beta * hv);
#pragma unroll
                for (int s = 1; s < 4; ++s) {
                    const float dg = d_grad ? d_grad[(int64_t)(s - 1) * n + j] : 0.0f;
                    zb[(int64_t)s * g.W + u] = w0 * dg;
                    gw0 = fmaf(dg, sg * h[(int64_t)s * g.W + u], gw0);
                }
            }
            gb0 += df;
            gb1 += dl;
        }
    }
    red[0][threadIdx.y][threadIdx.x] = gw0;
    red[1][threadIdx.y][threadIdx.x] = gw1;
    red[2][threadIdx.y][threadIdx.x] = gb0;
    red[3][threadIdx.y][threadIdx.x] = gb1;
    __syncthreads();
    if (threadIdx.y == 0 && u < g.W) {
        float t0 = 0.0f, t1 = 0.0f, b0 = 0.0f, b1 = 0.0f;
        for (int q = 0; q < 8; ++q) {
            t0 += red[0][q][threadIdx.x];
            t1 += red[1][q][threadIdx.x];
            b0 += red[2][q][threadIdx.x];
            b1 += red[3][q][threadIdx.x];
        }
        float* part = partial + (int64_t)sp * split_stride;
        part[g.off_w[g.NH] + u] = t0;
        if (g.head_out == 2) part[g.off_w[g.NH] + g.W + u] = t1;
        if (u == 0) {
            part[g.off_b[g.NH]] = b0;
            if (g.head_out == 2) part[g.off_b[g.NH] + 1] = b1;
        }
    }
}

// pre-activation adjoint in place (zbar -> hbar) and the bias partials:
// hb0 = zb0 sg + (sum_s zb_s h_s) beta sg (1 - sg), hb_s = sg zb_s.
// Block (split, 32-unit chunk): threadIdx.x = unit, threadIdx.y = one of 8
// point lanes; the lanes' bias sums are added in a fixed order.
__global__ void __launch_bounds__(256) whbar_kernel(WNet g, int l, int64_t n, int64_t pps,
                                                    const float* __restrict__ H, float* __restrict__ zbar,
                                                    float* __restrict__ partial, int64_t split_stride) {
    __shared__ float red[8][32];
    const int sp = blockIdx.x;
    const int u = blockIdx.y * 32 + threadIdx.x;
    const int64_t j0 = (int64_t)sp * pps, j1 = min(n, j0 + pps);
    float gb = 0.0f;
    if (u < g.W) {
#pragma unroll 2
        for (int64_t j = j0 + threadIdx.y; j < j1; j += 8) {
            const float* h = H + (j * g.S) * g.W;
            float* zb = zbar + (j * g.S) * g.W;
            const float hv = h[u];
            const float sg = sigm_w(g.beta * hv);
            float b0 = zb[u] * sg;
            if (g.S == 4) {
                const float ds = g.beta * sg * (1.0f - sg);
                float t = 0.0f;
#pragma unroll
                for (int s = 1; s < 4; ++s) {
                    const float z = zb[(int64_t)s * g.W + u];
                    t = fmaf(z, h[(int64_t)s * g.W + u], t);
                    zb[(int64_t)s * g.W + u] = sg * z;
                }
                b0 = fmaf(t, ds, b0);
            }
            zb[u] = b0;
            gb += b0;
        }
    }
    red[threadIdx.y][threadIdx.x] = gb;
    __syncthreads();
    if (threadIdx.y == 0 && u < g.W) {
        float t = 0.0f;
        for (int q = 0; q < 8; ++q) t += red[q][threadIdx.x];
        partial[(int64_t)sp * split_stride + g.off_b[l] + u] = t;
    }
}

// the per-split parameter-gradient partials summed in split order, Kahan
// compensated in FP32 (deterministic; FP64 is a small fraction of FP32 here)
__global__ void wreduce_partials(const float* __restrict__ partial, int n_split, int64_t stride, int64_t n,
                                 float* __restrict__ out) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    float acc = 0.0f, cmp = 0.0f;
    for (int c = 0; c < n_split; ++c) {
        const float y = partial[(int64_t)c * stride + i] - cmp;
        const float t = acc + y;
        cmp = (t - acc) - y;
        acc = t;
    }
    out[i] = acc - cmp;
}

inline unsigned gdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }

// ------------------------------------------------------------ host helpers
struct Nets {
    WNet sdf, refl;
    int two;            // 1: separate reflectivity network
    int64_t n_params;   // all packed parameters
};

bool make_nets(const geraf_field_desc* d, int S_sdf, Nets* nets) {
    nets->two = d->refl_hidden > 0;
    if (!make_wnet(d->params, d->n_levels, d->width, d->n_hidden, nets->two ? 1 : 2, S_sdf, d, &nets->sdf))
        return false;
    nets->n_params = nets->sdf.n_params;
    if (nets->two) {
        if (!make_wnet(d->params + nets->sdf.n_params, d->n_levels, d->refl_width, d->refl_hidden, 1, 1, d,
                       &nets->refl))
            return false;
        nets->n_params += nets->refl.n_params;
    }
    return true;
}

// saved layout: [SDF: Z0 (n S K0p) | H_0 .. H_{NH-1} (n S W each)] [refl: same with S = 1] [a (n)]
size_t net_floats(const WNet& g, int64_t n) { return (size_t)n * g.S * ((size_t)g.K0p + (size_t)g.NH * g.W); }

void net_forward(const WNet& g, const float* xyz, int64_t n, float* base, cudaStream_t st) {
    float* Z0 = base;
    wpe_kernel<<<gdiv(3 * n, 256), 256, 0, st>>>(xyz, n, g, Z0);
    const float* in = Z0;
    int64_t ld_in = g.K0p;
    float* H = Z0 + (size_t)n * g.S * g.K0p;
    for (int l = 0; l < g.NH; ++l) {
        WGemm p{};
        p.M = n * g.S;
        p.N = g.W;
        p.Kc = g.k_pad(l);
        p.a = in;
        p.lda = ld_in;
        p.b = g.params + g.off_w[l];
        p.ldb = g.k_in(l);
        p.act = l > 0;
        p.S = g.S;
        p.beta = g.beta;
        p.c = H;
        p.ldc = g.W;
        p.bias = g.params + g.off_b[l];
        wgemm_kernel<WG_FWD><<<dim3(gdiv(g.W, GN), gdiv(p.M, GM)), GT, wgemm_smem(), st>>>(p);
        in = H;
        ld_in = g.W;
        H += (size_t)n * g.S * g.W;
    }
}

}  // namespace

// ---------------------------------------------------------------- entry glue
bool mlp_is_wide(const geraf_field_desc* d) { return d->refl_hidden > 0 || d->width != 128; }

geraf_status mlp_wide_tc_saved_bytes(const geraf_field_desc* d, int64_t n, size_t* bytes);
geraf_status mlp_wide_tc_forward(const geraf_field_desc* d, const float* xyz, int64_t n, float* sdf, float* grad,
                                 float* refl, void* saved, size_t saved_bytes, cudaStream_t st);
geraf_status mlp_wide_tc_backward(const geraf_field_desc* d, const float* xyz, int64_t n, const void* saved,
                                  const float* d_sdf, const float* d_grad, const float* d_refl, float* d_params,
                                  void* ws, size_t* ws_bytes, cudaStream_t st);

geraf_status mlp_wide_saved_bytes(const geraf_field_desc* d, int64_t n, size_t* bytes) {
    if (d->precision == GERAF_PREC_BF16) return mlp_wide_tc_saved_bytes(d, n, bytes);
    Nets nets;
    if (!make_nets(d, 4, &nets)) return GERAF_ERR_UNSUPPORTED;
    size_t f = net_floats(nets.sdf, n) + (size_t)n;
    if (nets.two) f += net_floats(nets.refl, n);
    *bytes = f * sizeof(float);
    return GERAF_OK;
}

geraf_status mlp_wide_forward(const geraf_field_desc* d, const float* xyz, int64_t n, float* sdf, float* grad,
                              float* refl, void* saved, size_t saved_bytes, cudaStream_t st) {
    if (d->precision == GERAF_PREC_BF16)
        return mlp_wide_tc_forward(d, xyz, n, sdf, grad, refl, saved, saved_bytes, st);
    if (d->precision != GERAF_PREC_FP32)
        return fail(GERAF_ERR_UNSUPPORTED, "fields: MLP precision %d unknown", d->precision);
    if (!saved)
        return fail(GERAF_ERR_INVALID_ARG, "fields: this network keeps its layer activations in `saved`, which "
                                           "must be given even without a backward pass");
    size_t need = 0;
    geraf_status s0 = mlp_wide_saved_bytes(d, n, &need);
    if (s0 != GERAF_OK) return s0;
    if (saved_bytes < need) return fail(GERAF_ERR_WORKSPACE, "fields: saved %zu < %zu bytes", saved_bytes, need);
    // tangent streams only when the gradient is asked for
    Nets nets;
    if (!make_nets(d, grad ? 4 : 1, &nets)) return GERAF_ERR_UNSUPPORTED;
    {
        const geraf_status as = smem_attrs((int)wgemm_smem(), "shared-memory opt-in", wgemm_kernel<WG_FWD>,
                                           wgemm_kernel<WG_DZ>, wgemm_kernel<WG_DW>);
        if (as != GERAF_OK) return as;
    }
    Nets full;
    make_nets(d, 4, &full);
    float* base = static_cast<float*>(saved);
    float* a_saved = base + net_floats(full.sdf, n) + (full.two ? net_floats(full.refl, n) : 0);
    const WNet& gs = nets.sdf;
    net_forward(gs, xyz, n, base, st);
    const float* Hs = base + (size_t)n * gs.S * (gs.K0p + (size_t)(gs.NH - 1) * gs.W);
    whead_fwd_kernel<<<gdiv(n * 32, 256), 256, 0, st>>>(gs, n, Hs, sdf, grad, nets.two ? nullptr : refl,
                                                        nets.two ? nullptr : a_saved, nets.two ? -1 : 1);
    if (nets.two && refl) {
        // the reflectivity network (value stream only) behind the SDF network's
        // full four-stream block, so the layout matches the backward pass
        float* rb = base + net_floats(full.sdf, n);
        const WNet& gr = nets.refl;
        net_forward(gr, xyz, n, rb, st);
        const float* Hr = rb + (size_t)n * gr.S * (gr.K0p + (size_t)(gr.NH - 1) * gr.W);
        whead_fwd_kernel<<<gdiv(n * 32, 256), 256, 0, st>>>(gr, n, Hr, nullptr, nullptr, refl, a_saved, 0);
    }
    return cuda_status(cudaGetLastError(), "fields(wide mlp)");
}

namespace {
int wide_splits(int64_t n) {
    const int64_t s = (int64_t)device_sm_count() / 2;
    return (int)std::max<int64_t>(1, std::min<int64_t>(s, (n + 63) / 64));
}

void net_backward(const WNet& g, const float* xyz, int64_t n, const float* base, const float* a_saved,
                  const float* d_f, const float* d_grad, const float* d_a, int refl_net, float* zA, float* zB,
                  float* partial, int64_t split_stride, int splits, cudaStream_t st) {
    const int64_t pps = (n + splits - 1) / splits;
    const float* Z0 = base;
    const float* Hl = Z0 + (size_t)n * g.S * g.K0p;
    auto H_of = [&](int l) { return Hl + (size_t)l * n * g.S * g.W; };
    whead_bwd_kernel<<<dim3(splits, gdiv(g.W, 32)), dim3(32, 8), 0, st>>>(g, n, pps, H_of(g.NH - 1), a_saved, d_f,
                                                                        d_grad, d_a, refl_net, zA, partial,
                                                                        split_stride);
    const int64_t rows = n * g.S;
    const int64_t rps = (pps * g.S + GK - 1) / GK * GK;
    for (int l = g.NH - 1; l >= 0; --l) {
        whbar_kernel<<<dim3(splits, gdiv(g.W, 32)), dim3(32, 8), 0, st>>>(g, l, n, pps, H_of(l), zA, partial,
                                                                         split_stride);
        // weight gradient: partial[u][k] = sum over the split's rows of hb[r][u] z[r][k]
        WGemm w{};
        w.M = g.W;
        w.N = g.k_pad(l);
        w.a = zA;
        w.lda = g.W;
        w.b = l == 0 ? Z0 : H_of(l - 1);
        w.ldb = g.k_pad(l);
        w.act = l > 0;
        w.S = g.S;
        w.beta = g.beta;
        w.c = partial + g.off_w[l];
        w.ldc = g.k_in(l);
        w.n_valid = g.k_in(l);
        w.rows = rows;
        w.rows_per_split = rps;
        w.split_stride = split_stride;
        const int nsplit = (int)((rows + rps - 1) / rps);
        wgemm_kernel<WG_DW><<<dim3(gdiv(w.N, GN), gdiv(w.M, GM), nsplit), GT, wgemm_smem(), st>>>(w);
        if (l > 0) {
            // input adjoint: zB[r][k] = sum_u hb[r][u] W[u][k]
            WGemm z{};
            z.M = rows;
            z.N = g.W;
            z.Kc = g.W;
            z.a = zA;
            z.lda = g.W;
            z.b = g.params + g.off_w[l];
            z.ldb = g.W;
            z.S = g.S;
            z.c = zB;
            z.ldc = g.W;
            wgemm_kernel<WG_DZ><<<dim3(gdiv(z.N, GN), gdiv(z.M, GM)), GT, wgemm_smem(), st>>>(z);
            float* t = zA; zA = zB; zB = t;
        }
    }
}
}  // namespace

geraf_status mlp_wide_backward(const geraf_field_desc* d, const float* xyz, int64_t n, const void* saved,
                               const float* d_sdf, const float* d_grad, const float* d_refl, float* d_params,
                               void* ws, size_t* ws_bytes, cudaStream_t st) {
    if (d->precision == GERAF_PREC_BF16)
        return mlp_wide_tc_backward(d, xyz, n, saved, d_sdf, d_grad, d_refl, d_params, ws, ws_bytes, st);
    if (d->precision != GERAF_PREC_FP32)
        return fail(GERAF_ERR_UNSUPPORTED, "fields_backward: MLP precision %d unknown", d->precision);
    Nets nets;
    if (!make_nets(d, 4, &nets)) return GERAF_ERR_UNSUPPORTED;
    const int splits = wide_splits(n);
    // the DW kernel splits rows in chunks of whole tiles: at most as many splits as the head/bias kernels
    const int64_t wmax = std::max<int64_t>(std::max(nets.sdf.W, nets.sdf.K0p),
                                           nets.two ? std::max(nets.refl.W, nets.refl.K0p) : 0);
    WsCarver c(ws);
    float* zA = c.take<float>((size_t)n * 4 * wmax);
    float* zB = c.take<float>((size_t)n * 4 * wmax);
    float* partial = c.take<float>((size_t)splits * nets.n_params);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used)
        return fail(GERAF_ERR_WORKSPACE, "fields_backward: workspace %zu < %zu bytes", *ws_bytes, c.used);
    if (!saved) return fail(GERAF_ERR_INVALID_ARG, "fields_backward: saved is NULL");
    {
        const geraf_status as = smem_attrs((int)wgemm_smem(), "shared-memory opt-in", wgemm_kernel<WG_DZ>,
                                           wgemm_kernel<WG_DW>);
        if (as != GERAF_OK) return as;
    }
    // every split row of `partial` is written in full by the kernels below
    cudaError_t e = cudaMemsetAsync(partial, 0, (size_t)splits * nets.n_params * sizeof(float), st);
    if (e != cudaSuccess) return cuda_status(e, "fields_backward(wide mlp) memset");
    const float* base = static_cast<const float*>(saved);
    const float* a_saved = base + net_floats(nets.sdf, n) + (nets.two ? net_floats(nets.refl, n) : 0);
    net_backward(nets.sdf, xyz, n, base, a_saved, d_sdf, d_grad, nets.two ? nullptr : d_refl, 0, zA, zB, partial,
                 nets.n_params, splits, st);
    if (nets.two)
        net_backward(nets.refl, xyz, n, base + net_floats(nets.sdf, n), a_saved, nullptr, nullptr, d_refl, 1, zA,
                     zB, partial + nets.sdf.n_params, nets.n_params, splits, st);
    wreduce_partials<<<gdiv(nets.n_params, 256), 256, 0, st>>>(partial, splits, nets.n_params, nets.n_params,
                                                              d_params);
    return cuda_status(cudaGetLastError(), "fields_backward(wide mlp)");
}

}  // namespace geraf
