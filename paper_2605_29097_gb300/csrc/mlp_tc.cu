// BF16 SDF + reflectiveness MLP on the fifth-generation tensor cores
// (tcgen05): operands in shared memory (no-swizzle K-major BF16 tiles),
// accumulators in tensor memory (FP32), one elected thread issues the MMAs.
// A tile is 32 points x 4 streams (value, d/dx, d/dy, d/dz) = 128 columns;
// every hidden layer is D[128 units][128 columns] = W[128][K] X[K][128] with
// K = 16 * ceil(6L / 16) for the encoding layer and 128 after it. The
// epilogue reads D from tensor memory (tcgen05.ld), adds the bias, applies
// softplus to the value column and sigmoid(beta h) to the tangents, saves the
// FP32 pre-activations for the adjoint and writes the next layer's BF16
// operand. The head (f, a_logit, G = W_f dz) runs on CUDA cores in FP32 from
// the last BF16 activations.
#include <cuda_bf16.h>
#include <math.h>

#include "tcgen05.cuh"

namespace geraf {

namespace {

constexpr int TW = 128;          // hidden width
constexpr int TTP = 32;          // points per tile
constexpr int TCOL = 128;        // columns per tile
constexpr int TTHREADS = 128;
constexpr uint32_t TLBO = 128;   // K-direction core-matrix stride (bytes)

struct TcGeom {
    int L, K0, K0p, NH;
    float beta, cx, cy, cz, half;
    int64_t n;
    int n_tiles;
    int64_t off_w[8], off_b[8];
    float wk[21];       // 2^k pi / half: the encoding's x-derivative factors, per octave
};

bool make_tc_geom(const geraf_field_desc* d, int64_t n, TcGeom* g) {
    if (d->width != TW || d->n_levels < 1 || 6 * d->n_levels > TW || d->n_hidden < 1 || d->n_hidden > 4 ||
        !(d->half > 0.0f)) {
        set_error("fields(bf16): need width 128, 1 <= n_levels <= 21, 1 <= n_hidden <= 4");
        return false;
    }
    g->L = d->n_levels;
    g->K0 = 6 * d->n_levels;
    g->K0p = (g->K0 + 15) / 16 * 16;
    g->NH = d->n_hidden;
    g->beta = d->beta;
    g->cx = d->center[0]; g->cy = d->center[1]; g->cz = d->center[2];
    g->half = d->half;
    for (int k = 0; k < g->L; ++k) g->wk[k] = (float)((double)(1 << k) * 3.14159265358979323846 / (double)g->half);
    g->n = n;
    g->n_tiles = (int)((n + TTP - 1) / TTP);
    int64_t off = 0;
    for (int l = 0; l <= g->NH; ++l) {
        const int kin = l == 0 ? g->K0 : TW;
        const int out = l == g->NH ? 2 : TW;
        g->off_w[l] = off; off += (int64_t)out * kin;
        g->off_b[l] = off; off += out;
    }
    return true;
}

__device__ __forceinline__ float sgm(float x) { return 1.0f / (1.0f + expf(-x)); }

// softplus_beta(h) = max(h, 0) + log1p(e) / beta and sigmoid(beta h) from one
// exponential e = exp(-beta |h|): sigmoid(beta h) = 1 / (1 + e) for h >= 0 and
// e / (1 + e) below. One SFU exponential, one reciprocal and log1p per
// element instead of two exponentials, a logarithm and two divides. The
// forward and both adjoint recomputations call this same function, so the
// adjoint's BF16 layer inputs are bit for bit the operands the forward used.
__device__ __forceinline__ void act_pair(float h, float beta, float inv_beta, float& sp, float& sg) {
    const float e = __expf(-beta * fabsf(h));
    const float r = __fdividef(1.0f, 1.0f + e);
    sg = h >= 0.0f ? r : e * r;
    sp = fmaf(log1pf(e), inv_beta, fmaxf(h, 0.0f));
}

__device__ __forceinline__ void st_bf16(unsigned char* base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}
__device__ __forceinline__ float bf16r(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }

// Encoding features of axis d of point x (FP32 coordinate) and their
// x-derivatives: put(feature, stream, value) for stream 0 (value) and the
// three tangent streams (only stream d + 1 is nonzero).
template <class Put>
__device__ __forceinline__ void encode_axis(const TcGeom& g, float x, int d, Put put) {
    const float c = d == 0 ? g.cx : (d == 1 ? g.cy : g.cz);
    const double xt_ = ((double)x - (double)c) / (double)g.half;
    for (int k = 0; k < g.L; ++k) {
        const double t2 = xt_ * (double)(1 << k);
        const double r = t2 - 2.0 * rint(0.5 * t2);
        float sn, cs;
        sincospif((float)r, &sn, &cs);
        const float wk = g.wk[k];
        const int fs = 6 * k + d, fc = 6 * k + 3 + d;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            float vs, vc;
            if (s == 0) { vs = sn; vc = cs; }
            else if (s - 1 == d) { vs = wk * cs; vc = -wk * sn; }
            else { vs = 0.0f; vc = 0.0f; }
            put(fs, s, vs);
            put(fc, s, vc);
        }
    }
}

struct TcFwdArgs {
    TcGeom g;
    const float* params;
    const float* xyz;
    float* sdf;
    float* grad;
    float* refl;
    float* saved;     // [NH][n][4][128] FP32 pre-activations, then a[n]; may be null
    int* err;
};

// 8x8 transpose of 16-bit values across the 8 lanes of each aligned group of
// 8 lanes: on entry lane i of the group holds row i (p[k] = elements 2k and
// 2k + 1, the first in the low half), on exit it holds column i. Three
// exchange stages between lanes i and i ^ 4, i ^ 2, i ^ 1.
__device__ __forceinline__ void transpose8x8_b16(uint32_t (&p)[4]) {
    const int i = threadIdx.x & 7;
    {
        const bool hi = (i & 4) != 0;
        uint32_t s0 = hi ? p[0] : p[2], s1 = hi ? p[1] : p[3];
        s0 = __shfl_xor_sync(0xffffffffu, s0, 4);
        s1 = __shfl_xor_sync(0xffffffffu, s1, 4);
        if (hi) { p[0] = s0; p[1] = s1; } else { p[2] = s0; p[3] = s1; }
    }
    {
        const bool hi = (i & 2) != 0;
        uint32_t s0 = hi ? p[0] : p[1], s1 = hi ? p[2] : p[3];
        s0 = __shfl_xor_sync(0xffffffffu, s0, 2);
        s1 = __shfl_xor_sync(0xffffffffu, s1, 2);
        if (hi) { p[0] = s0; p[2] = s1; } else { p[1] = s0; p[3] = s1; }
    }
    {
        const bool hi = (i & 1) != 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint32_t w = __shfl_xor_sync(0xffffffffu, p[k], 1);
            p[k] = hi ? ((p[k] & 0xFFFF0000u) | (w >> 16)) : ((p[k] & 0xFFFFu) | (w << 16));
        }
    }
}

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
    const uint32_t a = __bfloat16_as_ushort(__float2bfloat16_rn(lo));
    const uint32_t b = __bfloat16_as_ushort(__float2bfloat16_rn(hi));
    return a | (b << 16);
}

constexpr int FTHREADS = 512;     // 16 warps: 4 TMEM lane quarters x 4 column chunks of 32

// Forward, two 32-point tiles in flight per CTA (accumulators in TMEM columns
// 0..127 and 128..255): while the epilogue of one tile runs, the MMAs of the
// other execute. Epilogue: warp w reads TMEM lanes 32 (w % 4) .. + 31 (units)
// and columns 32 (w / 4) .. + 31 (8 points x 4 streams) of its tile, adds the
// bias, applies softplus / sigmoid(beta h), saves the FP32 pre-activations and
// writes the next BF16 operand as 16-byte rows (one 8x8 transpose per block
// of 8 columns across each group of 8 lanes).
__global__ void __launch_bounds__(FTHREADS, 1) mlp_tc_fwd_kernel(const TcFwdArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcGeom& g = a.g;
    const float inv_beta = 1.0f / g.beta;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    unsigned char* wt[4];
    uint32_t off = 0;
    for (int l = 0; l < g.NH; ++l) {
        wt[l] = smem + off;
        off += (uint32_t)TW * (l == 0 ? g.K0p : TW) * 2u;
    }
    off = (off + 1023u) & ~1023u;
    unsigned char* xt[2] = {smem + off, smem + off + TCOL * TW * 2u};   // [128 columns][128 K] BF16 each
    off += 2u * TCOL * TW * 2u;
    float* bias = reinterpret_cast<float*>(smem + off);    // [NH][128]
    off += g.NH * TW * 4u;
    float* head = reinterpret_cast<float*>(smem + off);    // W_f[128], W_a[128], b_f, b_a
    off += (2 * TW + 2) * 4u;
    off = (off + 7u) & ~7u;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + off);           // [2]
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + off + 16);
    int* abort_flag = reinterpret_cast<int*>(smem + off + 20);

    for (int l = 0; l < g.NH; ++l) {
        const int K = l == 0 ? g.K0 : TW, Kp = l == 0 ? g.K0p : TW;
        const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
        const float* W = a.params + g.off_w[l];
        for (int i = t; i < TW * Kp; i += FTHREADS) {
            const int u = i / Kp, k = i - u * Kp;
            st_bf16(wt[l], tc::kmajor_offset(u, k, TLBO, sbo), k < K ? W[u * K + k] : 0.0f);
        }
        for (int i = t; i < TW; i += FTHREADS) bias[l * TW + i] = a.params[g.off_b[l] + i];
    }
    for (int i = t; i < 2 * TW; i += FTHREADS) head[i] = a.params[g.off_w[g.NH] + i];
    if (t < 2) head[2 * TW + t] = a.params[g.off_b[g.NH] + t];
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, TCOL);
    uint32_t phase[2] = {0u, 0u};
    bool pending[2] = {false, false};
    const int lq = warp & 3, cc = warp >> 2;
    const int u = 32 * lq + lane;                         // unit = TMEM lane
    const int n_pairs = (g.n_tiles + 1) / 2;

    auto issue = [&](int s, int l) {                      // thread 0: layer l of tile slot s
        const int Kp = l == 0 ? g.K0p : TW;
        const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
        const uint32_t wa = smem_u32(wt[l]), xa = smem_u32(xt[s]);
        for (int q = 0; q < Kp / 16; ++q)
            tc::mma_bf16(tbase + 128u * s, tc::smem_desc(wa + q * 256u, TLBO, sbo),
                         tc::smem_desc(xa + q * 256u, TLBO, sbo), idesc, q > 0 ? 1u : 0u);
        tc::mma_commit(&bar[s]);
    };

    for (int pair = blockIdx.x; pair < n_pairs; pair += gridDim.x) {
        const int nslot = (2 * pair + 1 < g.n_tiles) ? 2 : 1;
        // encoding of both tiles -> X (BF16, K = K0p; padding columns zero)
        {
            const uint32_t sbo0 = (uint32_t)(g.K0p / 8) * 128u;
            const int padw = g.K0p - g.K0;
            for (int i = t; i < nslot * TCOL * padw; i += FTHREADS) {
                const int s = i / (TCOL * padw), r = i - s * TCOL * padw;
                const int c = r / padw, k = g.K0 + r % padw;
                st_bf16(xt[s], tc::kmajor_offset(c, k, TLBO, sbo0), 0.0f);
            }
            if (t < nslot * 3 * TTP) {
                const int s = t / (3 * TTP), r = t - s * 3 * TTP;
                const int p = r / 3, d = r - 3 * (r / 3);
                int64_t j = (int64_t)(2 * pair + s) * TTP + p;
                if (j >= g.n) j = g.n - 1;
                encode_axis(g, a.xyz[d * g.n + j], d, [&](int f, int st, float v) {
                    st_bf16(xt[s], tc::kmajor_offset(4 * p + st, f, TLBO, sbo0), v);
                });
            }
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (t == 0)
            for (int s = 0; s < nslot; ++s) issue(s, 0);
        for (int s = 0; s < nslot; ++s) pending[s] = true;
        for (int l = 0; l < g.NH && !*abort_flag; ++l) {
            for (int s = 0; s < nslot; ++s) {
                const bool ok = mbar_wait(&bar[s], phase[s]);
                if (ok) phase[s] ^= 1u;
                pending[s] = !ok;                 // a timed-out MMA is still in flight
                if (!ok) atomicOr(abort_flag, 1);
                tc::fence_after_sync();
                __syncthreads();
                if (*abort_flag) break;
                const int64_t j0 = (int64_t)(2 * pair + s) * TTP;
                float r[32];
                tc::tmem_ld32(tbase + 128u * s + ((uint32_t)(32 * lq) << 16) + (uint32_t)(32 * cc), r);
                const float bu = bias[l * TW + u];
                float v[32];
#pragma unroll
                for (int pp = 0; pp < 8; ++pp) {
                    const float h = r[4 * pp] + bu;
                    float sg;
                    act_pair(h, g.beta, inv_beta, v[4 * pp], sg);
                    v[4 * pp + 1] = sg * r[4 * pp + 1];
                    v[4 * pp + 2] = sg * r[4 * pp + 2];
                    v[4 * pp + 3] = sg * r[4 * pp + 3];
                    const int64_t j = j0 + 8 * cc + pp;
                    if (a.saved && j < g.n) {
                        float* dst = a.saved + (((int64_t)l * g.n + j) * 4) * TW + u;
                        dst[0] = h;
                        dst[TW] = r[4 * pp + 1];
                        dst[2 * TW] = r[4 * pp + 2];
                        dst[3 * TW] = r[4 * pp + 3];
                    }
                }
                // next operand: 4 blocks of 8 columns, each an 8x8 transpose over 8 lanes
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    uint32_t q[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k) q[k] = pack_bf16x2(v[8 * b + 2 * k], v[8 * b + 2 * k + 1]);
                    transpose8x8_b16(q);
                    const int c = 32 * cc + 8 * b + (lane & 7);
                    const int u0 = 32 * lq + 8 * (lane >> 3);
                    *reinterpret_cast<uint4*>(xt[s] + tc::kmajor_offset(c, u0, TLBO, 16u * 128u)) =
                        make_uint4(q[0], q[1], q[2], q[3]);
                }
                tc::fence_async_smem();
                tc::fence_before_sync();
                __syncthreads();
                tc::fence_after_sync();
                if (l + 1 < g.NH) {
                    if (t == 0) issue(s, l + 1);
                    pending[s] = true;
                }
            }
        }
        if (*abort_flag) break;
        // head from the last BF16 activations of both tiles, thread = (tile, column)
        if (t < nslot * TCOL) {
            const int s = t / TCOL, c = t - s * TCOL, p = c >> 2, st = c & 3;
            const int64_t j = (int64_t)(2 * pair + s) * TTP + p;
            float v0 = 0.0f, v1 = 0.0f;
            for (int u8 = 0; u8 < TW; u8 += 8) {
                const uint4 raw = *reinterpret_cast<const uint4*>(xt[s] + tc::kmajor_offset(c, u8, TLBO, 16u * 128u));
                const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float x = __bfloat162float(e[q]);
                    v0 = fmaf(head[u8 + q], x, v0);
                    v1 = fmaf(head[TW + u8 + q], x, v1);
                }
            }
            if (j < g.n) {
                if (st == 0) {
                    a.sdf[j] = v0 + head[2 * TW];
                    const float av = sgm(v1 + head[2 * TW + 1]);
                    if (a.refl) a.refl[j] = av;
                    if (a.saved) a.saved[(int64_t)g.NH * g.n * 4 * TW + j] = av;
                } else if (a.grad) {
                    a.grad[(int64_t)(st - 1) * g.n + j] = v0;
                }
            }
        }
        __syncthreads();   // the next pair's encoding overwrites the tiles the head read
    }
    if (*abort_flag && t == 0) {
        atomicOr(a.err, 1);
        for (int s = 0; s < 2; ++s)      // bounded: let timed-out or issued MMAs finish before TMEM is freed
            if (pending[s]) mbar_wait(&bar[s], phase[s], 100000000ull);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

size_t tc_fwd_smem(const TcGeom& g) {
    size_t off = 0;
    for (int l = 0; l < g.NH; ++l) off += (size_t)TW * (l == 0 ? g.K0p : TW) * 2;
    off = (off + 1023) & ~(size_t)1023;
    off += 2 * TCOL * TW * 2;
    off += g.NH * TW * 4 + (2 * TW + 2) * 4;
    off = (off + 7) & ~(size_t)7;
    return off + 24 + 1024;   // barriers, TMEM slot, abort flag; slack for the 1024-byte base alignment
}

// ------------------------------------------------------- adjoint (BF16 network)
// Straight-through adjoint of the BF16 network: each rounding passes as the
// identity, so the products use the operands the forward multiplied (BF16
// weights, BF16 layer inputs and tangents); the head weights are FP32.
// Hidden layer, per tile of 16 points (64 columns = 16 points x 4 streams):
//   Hb[c][u]  pre-activation adjoint in FP32 from the activation adjoint and
//             the saved pre-activations, split into BF16 hi + lo;
//   dW[u][k] += sum_c Hb[c][u] Z[c][k]: M = 128 units, N = K_in, K = 64
//             columns, accumulated in TMEM over all the CTA's tiles;
//   Z'[k][c]  = sum_u W[u][k] Hb[c][u] (the adjoint of the layer input,
//             transposed: M = K_in, N = 64, K = 128), read back per tile and
//             written over the activation adjoint.
// Every product is hi + lo of Hb against exact BF16 operands: 2 MMAs each.
constexpr int BTP = 16;          // points per adjoint tile
constexpr int BCOL = 4 * BTP;    // 64 columns
constexpr uint32_t B_SBO_K128 = 16u * 128u;   // 8-row group stride of a K = 128 tile
constexpr uint32_t B_SBO_K64 = 8u * 128u;     // 8-row group stride of a K = 64 tile

struct TcBwdArgs {
    TcGeom g;
    const float* params;
    const float* xyz;
    const float* saved;     // [NH][n][4][128] FP32 pre-activations, then a[n]
    const float* d_sdf;
    const float* d_grad;
    const float* d_refl;
    float* zbar;            // [n][4][128] activation adjoint, updated layer by layer
    float* partial;         // [gridDim.x][n_params]
    int64_t n_params;
    int layer;
    int* err;
};

// head: dL/dW_head, dL/db_head (from the BF16-rounded last activations) and
// the adjoint of the last hidden activation (through the FP32 head weights);
// thread = (unit, point slot of HB_SLOTS), R points per slot in flight
constexpr int HB_SLOTS = 8;
constexpr int HB_THREADS = HB_SLOTS * TW;
__global__ void __launch_bounds__(HB_THREADS) mlp_tc_head_bwd_kernel(const TcBwdArgs a) {
    __shared__ float red[2 * HB_THREADS];
    __shared__ float redb[2 * HB_SLOTS];
    const TcGeom& g = a.g;
    const int t = threadIdx.x, u = t & (TW - 1), half = t >> 7;   // half: the thread's point slot
    const float* Wh = a.params + g.off_w[g.NH];
    const float w0 = Wh[u], w1 = Wh[TW + u];
    const float* hsv = a.saved + (int64_t)(g.NH - 1) * g.n * 4 * TW;
    const float* asv = a.saved + (int64_t)g.NH * g.n * 4 * TW;
    float gw0 = 0.0f, gw1 = 0.0f, gb0 = 0.0f, gb1 = 0.0f;
    constexpr int R = 4;                                   // points per thread per round, loads in flight
    for (int64_t base = (int64_t)blockIdx.x * HB_SLOTS * R; base < g.n;
         base += (int64_t)gridDim.x * HB_SLOTS * R) {
        float df[R], dl[R], dG[R][3], h0[R], hd[R][3];
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t j = base + HB_SLOTS * r + half;
            const bool ok = j < g.n;
            const int64_t jj = ok ? j : 0;
            const float* h = hsv + jj * 4 * TW;
            df[r] = ok && a.d_sdf ? a.d_sdf[jj] : 0.0f;
            const float av = asv[jj];
            dl[r] = ok && a.d_refl ? a.d_refl[jj] * av * (1.0f - av) : 0.0f;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                dG[r][d] = ok && a.d_grad ? a.d_grad[(int64_t)d * g.n + jj] : 0.0f;
                hd[r][d] = h[(d + 1) * TW + u];
            }
            h0[r] = h[u];
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            const int64_t j = base + HB_SLOTS * r + half;
            if (j >= g.n) continue;
            float z, sg;
            act_pair(h0[r], g.beta, 1.0f / g.beta, z, sg);
            z = bf16r(z);
            gw0 += df[r] * z;
            gw1 += dl[r] * z;
            float* zb = a.zbar + j * 4 * TW;
            zb[u] = w0 * df[r] + w1 * dl[r];
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                gw0 += dG[r][d] * bf16r(sg * hd[r][d]);
                zb[(d + 1) * TW + u] = w0 * dG[r][d];
            }
            if (u == 0) { gb0 += df[r]; gb1 += dl[r]; }
        }
    }
    red[t] = gw0;
    red[HB_THREADS + t] = gw1;
    if (u == 0) { redb[2 * half] = gb0; redb[2 * half + 1] = gb1; }
    __syncthreads();
    float* out = a.partial + (int64_t)blockIdx.x * a.n_params;
    if (t < TW) {                                     // slots added in a fixed order
        float s0 = 0.0f, s1 = 0.0f;
        for (int q = 0; q < HB_SLOTS; ++q) {
            s0 += red[q * TW + t];
            s1 += red[HB_THREADS + q * TW + t];
        }
        out[g.off_w[g.NH] + t] = s0;
        out[g.off_w[g.NH] + TW + t] = s1;
    }
    if (t == 0) {
        float b0 = 0.0f, b1 = 0.0f;
        for (int q = 0; q < HB_SLOTS; ++q) {
            b0 += redb[2 * q];
            b1 += redb[2 * q + 1];
        }
        out[g.off_b[g.NH]] = b0;
        out[g.off_b[g.NH] + 1] = b1;
    }
}

struct BwdLayout {
    uint32_t wt, hbB, hbA, zB, zs, hsb, zin, bar;
    uint32_t total;
};

__host__ __device__ inline BwdLayout bwd_layout(int kin) {
    BwdLayout L;
    uint32_t off = 0;
    L.wt = off;  off += (uint32_t)kin * TW * 2u;            // W^T: rows k, K = 128 units
    L.hbB = off; off += 2u * BCOL * TW * 2u;                // Hb hi, lo: rows c, K = 128 units
    L.hbA = off; off += 2u * TW * BCOL * 2u;                // Hb hi, lo: rows u, K = 64 columns
    L.zB = off;  off += (uint32_t)kin * BCOL * 2u;          // Z: rows k, K = 64 columns
    L.zs = off;  off += BCOL * TW * 4u;                     // FP32 staging [64][128]
    L.hsb = off; off += BCOL * TW * 4u;                     // FP32 staging [64][128]
    L.zin = off; off += BCOL * TW * 4u;                     // FP32 staging [64][128]: the layer input's pre-activations
    L.bar = off; off += 16u + 4u * TW * 4u;                 // barrier, TMEM slot, abort flag, bias partials
    L.total = off;
    return L;
}

// Rows c = 4 p + s of a [n][4][128] FP32 array for points j0 + p (p < 16)
// into a [64][128] shared tile, all in flight; rows of points >= n read as 0.
__device__ __forceinline__ void stage64(float* dst, const float* src, int64_t j0, int64_t n) {
    for (int i = threadIdx.x; i < BCOL * (TW / 4); i += blockDim.x) {
        const int c = i >> 5, q = i & 31;
        const bool ok = j0 + (c >> 2) < n;
        cp_async16(dst + c * TW + 4 * q, ok ? src + (j0 * 4 + c) * TW + 4 * q : src, ok ? 16 : 0);
    }
}

constexpr int BTHREADS = 512;    // 16 warps: thread = (unit, chunk of 4 points); warp = (lane quarter, chunk)

__global__ void __launch_bounds__(BTHREADS, 1) mlp_tc_layer_bwd_kernel(const TcBwdArgs a) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char* smem = smem_raw;
    const TcGeom& g = a.g;
    const float inv_beta = 1.0f / g.beta;
    const int li = a.layer;
    const int kin = li == 0 ? g.K0p : TW;     // padded input width (MMA N of dW, M of the input adjoint)
    const int K = li == 0 ? g.K0 : TW;        // true input width
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int uu = t & (TW - 1);              // unit (Hb) or input unit (Z) of this thread
    const int ch = t >> 7;                    // chunk: points 4 ch .. 4 ch + 3 = columns 16 ch .. 16 ch + 15
    const int lq = warp & 3;                  // TMEM lane quarter of this warp (lanes 32 lq .. + 31)
    const BwdLayout L = bwd_layout(kin);
    unsigned char* wt = smem + L.wt;
    unsigned char* hbB[2] = {smem + L.hbB, smem + L.hbB + BCOL * TW * 2};
    unsigned char* hbA[2] = {smem + L.hbA, smem + L.hbA + TW * BCOL * 2};
    unsigned char* zB = smem + L.zB;
    float* zs = reinterpret_cast<float*>(smem + L.zs);
    float* hsb = reinterpret_cast<float*>(smem + L.hsb);
    float* zin = reinterpret_cast<float*>(smem + L.zin);
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + L.bar);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + L.bar + 8);
    int* abort_flag = reinterpret_cast<int*>(smem + L.bar + 12);
    float* redb = reinterpret_cast<float*>(smem + L.bar + 16);     // [4][128] bias partials

    // W^T as the A operand of the input adjoint (layers above the first)
    if (li > 0) {
        const float* W = a.params + g.off_w[li];      // [128 u][128 k]
        for (int i = t; i < TW * TW; i += BTHREADS) {
            const int u = i / TW, k = i - u * TW;
            st_bf16(wt, tc::kmajor_offset(k, u, TLBO, B_SBO_K128), W[i]);
        }
    } else {
        // padding rows K0 .. K0p-1 of Z stay zero for every tile
        for (int i = t; i < (kin - K) * BCOL; i += BTHREADS) {
            const int k = K + i / BCOL, c = i % BCOL;
            st_bf16(zB, tc::kmajor_offset(k, c, TLBO, B_SBO_K64), 0.0f);
        }
    }
    if (t == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t t_dw = tbase, t_dx = tbase + 128u;   // dW: columns 0..kin-1; input adjoint: 128..191
    const uint32_t id_dw = tc::idesc_bf16(128, kin);
    const uint32_t id_dx = tc::idesc_bf16(128, BCOL);
    const float* hs = a.saved + (int64_t)li * g.n * 4 * TW;
    const float* hin = li > 0 ? a.saved + (int64_t)(li - 1) * g.n * 4 * TW : nullptr;
    const int n_tiles = (int)((g.n + BTP - 1) / BTP);
    uint32_t phase = 0;
    bool pending = false;
    float accb = 0.0f;
    bool first = true;

    // the tile's three FP32 inputs (activation adjoint, this layer's and the
    // layer below's pre-activations), all in flight; the next tile's are
    // issued while this tile's MMAs, read-back and stores run
    auto stage_tile = [&](int64_t jt) {
        stage64(zs, a.zbar, jt, g.n);
        stage64(hsb, hs, jt, g.n);
        if (hin) stage64(zin, hin, jt, g.n);
    };
    if (blockIdx.x < n_tiles) stage_tile((int64_t)blockIdx.x * BTP);
    for (int tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
        const int64_t j0 = (int64_t)tile * BTP;
        cp_async_wait_all();
        __syncthreads();
        // pre-activation adjoint of unit uu for 4 points: 16 columns, hi and lo
        {
            float bv[16];
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const int c0 = 16 * ch + 4 * pp;
                const float* z = zs + c0 * TW + uu;
                const float* h = hsb + c0 * TW + uu;
                const float h0 = h[0];
                float sp_unused, sg;
                act_pair(h0, g.beta, inv_beta, sp_unused, sg);
                const float dsg = g.beta * sg * (1.0f - sg);
                const float z0 = z[0], z1 = z[TW], z2 = z[2 * TW], z3 = z[3 * TW];
                bv[4 * pp] = z0 * sg + (z1 * h[TW] + z2 * h[2 * TW] + z3 * h[3 * TW]) * dsg;
                bv[4 * pp + 1] = sg * z1;
                bv[4 * pp + 2] = sg * z2;
                bv[4 * pp + 3] = sg * z3;
                accb += bv[4 * pp];                   // 0 for points >= n (staged zeros)
            }
            uint32_t qh[8], ql[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const float h0v = bf16r(bv[2 * k]), h1v = bf16r(bv[2 * k + 1]);
                qh[k] = pack_bf16x2(h0v, h1v);
                ql[k] = pack_bf16x2(bv[2 * k] - h0v, bv[2 * k + 1] - h1v);
            }
            // A operand of dW: row uu, columns 16 ch .. + 15 as two 16-byte rows
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const uint32_t o = tc::kmajor_offset(uu, 16 * ch + 8 * hh, TLBO, B_SBO_K64);
                *reinterpret_cast<uint4*>(hbA[0] + o) = make_uint4(qh[4 * hh], qh[4 * hh + 1], qh[4 * hh + 2], qh[4 * hh + 3]);
                *reinterpret_cast<uint4*>(hbA[1] + o) = make_uint4(ql[4 * hh], ql[4 * hh + 1], ql[4 * hh + 2], ql[4 * hh + 3]);
            }
            // B operand of the input adjoint: rows = columns, 8 units per 16 bytes (8x8 transpose over 8 lanes)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                uint32_t th[4] = {qh[4 * hh], qh[4 * hh + 1], qh[4 * hh + 2], qh[4 * hh + 3]};
                uint32_t tl[4] = {ql[4 * hh], ql[4 * hh + 1], ql[4 * hh + 2], ql[4 * hh + 3]};
                transpose8x8_b16(th);
                transpose8x8_b16(tl);
                const int c = 16 * ch + 8 * hh + (lane & 7);
                const int u0 = uu & ~7;
                const uint32_t o = tc::kmajor_offset(c, u0, TLBO, B_SBO_K128);
                *reinterpret_cast<uint4*>(hbB[0] + o) = make_uint4(th[0], th[1], th[2], th[3]);
                *reinterpret_cast<uint4*>(hbB[1] + o) = make_uint4(tl[0], tl[1], tl[2], tl[3]);
            }
        }
        // the layer's BF16 input Z (thread = input unit uu, 4 points), as the forward rounded it
        if (hin) {
            uint32_t q[8];
#pragma unroll
            for (int pp = 0; pp < 4; ++pp) {
                const float* x = zin + (16 * ch + 4 * pp) * TW + uu;
                const float x0 = x[0];
                float z0, s0;
                act_pair(x0, g.beta, inv_beta, z0, s0);
                q[2 * pp] = pack_bf16x2(z0, s0 * x[TW]);
                q[2 * pp + 1] = pack_bf16x2(s0 * x[2 * TW], s0 * x[3 * TW]);
            }
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
                *reinterpret_cast<uint4*>(zB + tc::kmajor_offset(uu, 16 * ch + 8 * hh, TLBO, B_SBO_K64)) =
                    make_uint4(q[4 * hh], q[4 * hh + 1], q[4 * hh + 2], q[4 * hh + 3]);
        } else if (t < 3 * BTP) {
            const int p = t / 3, d = t - 3 * (t / 3);
            int64_t j = j0 + p;
            if (j >= g.n) j = g.n - 1;
            encode_axis(g, a.xyz[d * g.n + j], d, [&](int f, int s, float v) {
                st_bf16(zB, tc::kmajor_offset(f, 4 * p + s, TLBO, B_SBO_K64), v);
            });
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        // the staging buffers are consumed: the next tile's inputs may land
        if (tile + (int)gridDim.x < n_tiles) stage_tile((int64_t)(tile + gridDim.x) * BTP);
        if (t == 0) {
            const uint32_t zb_a = smem_u32(zB);
            for (int h = 0; h < 2; ++h) {
                const uint32_t ha = smem_u32(hbA[h]);
                for (int s = 0; s < BCOL / 16; ++s)
                    tc::mma_bf16(t_dw, tc::smem_desc(ha + s * 256u, TLBO, B_SBO_K64),
                                 tc::smem_desc(zb_a + s * 256u, TLBO, B_SBO_K64), id_dw,
                                 (!first || h > 0 || s > 0) ? 1u : 0u);
            }
            if (li > 0) {
                const uint32_t wa = smem_u32(wt);
                for (int h = 0; h < 2; ++h) {
                    const uint32_t hb = smem_u32(hbB[h]);
                    for (int s = 0; s < TW / 16; ++s)
                        tc::mma_bf16(t_dx, tc::smem_desc(wa + s * 256u, TLBO, B_SBO_K128),
                                     tc::smem_desc(hb + s * 256u, TLBO, B_SBO_K128), id_dx,
                                     (h > 0 || s > 0) ? 1u : 0u);
                }
            }
            tc::mma_commit(bar);
        }
        first = false;
        const bool ok = mbar_wait(bar, phase);
        if (ok) phase ^= 1u;
        pending = !ok;
        if (!ok) atomicOr(abort_flag, 1);
        tc::fence_after_sync();
        __syncthreads();
        if (*abort_flag) break;
        // adjoint of the layer input: warp = (lane quarter lq: input units, chunk ch: 16 columns)
        if (li > 0) {
            const int k = 32 * lq + lane;
            float r[16];
            tc::tmem_ld16(t_dx + ((uint32_t)(32 * lq) << 16) + (uint32_t)(16 * ch), r);
#pragma unroll
            for (int i = 0; i < 16; ++i) {
                const int c = 16 * ch + i;
                if (j0 + (c >> 2) < g.n) a.zbar[(j0 * 4 + c) * TW + k] = r[i];
            }
        }
        tc::fence_before_sync();
        __syncthreads();     // the next tile's staging and operands overwrite this tile's
    }
    cp_async_wait_all();      // a prefetch left in flight by an abort lands before the CTA exits
    redb[ch * TW + uu] = accb;
    if (*abort_flag) {
        if (t == 0) {
            atomicOr(a.err, 1);
            if (pending) mbar_wait(bar, phase, 100000000ull);   // bounded: let the timed-out MMAs finish
        }
    } else {
        // weight gradient of this CTA: warp = (lane quarter: units, chunk: 32 input columns)
        const int u = 32 * lq + lane;
        float* out = a.partial + (int64_t)blockIdx.x * a.n_params;
        if (32 * ch < kin) {
            float r[32];
            tc::tmem_ld32(t_dw + ((uint32_t)(32 * lq) << 16) + (uint32_t)(32 * ch), r);
#pragma unroll
            for (int i = 0; i < 32; ++i) {
                const int k = 32 * ch + i;
                if (k < K) out[g.off_w[li] + (int64_t)u * K + k] = first ? 0.0f : r[i];
            }
        }
    }
    __syncthreads();
    if (!*abort_flag && t < TW) {
        float* out = a.partial + (int64_t)blockIdx.x * a.n_params;
        out[g.off_b[li] + t] = ((redb[t] + redb[TW + t]) + redb[2 * TW + t]) + redb[3 * TW + t];
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

}  // namespace

geraf_status mlp_tc_forward_impl(const geraf_field_desc* d, const float* xyz, int64_t n, float* sdf, float* grad,
                                 float* refl, void* saved, cudaStream_t st) {
    TcGeom g;
    if (!make_tc_geom(d, n, &g)) return GERAF_ERR_UNSUPPORTED;
    const size_t smem = tc_fwd_smem(g);
    {
        const geraf_status as = smem_attrs(227 * 1024, "shared-memory opt-in", mlp_tc_fwd_kernel);
        if (as != GERAF_OK) return as;
    }
    int n_cta = device_sm_count();
    if (n_cta > (g.n_tiles + 1) / 2) n_cta = (g.n_tiles + 1) / 2;
    TcFwdArgs a{g, d->params, xyz, sdf, grad, refl, static_cast<float*>(saved), device_error_word()};
    mlp_tc_fwd_kernel<<<n_cta, FTHREADS, smem, st>>>(a);
    return cuda_status(cudaGetLastError(), "fields(mlp bf16)");
}

int mlp_tc_backward_ctas(int64_t n) {
    const int64_t tiles = (n + BTP - 1) / BTP;
    const int sms = device_sm_count();
    return (int)(tiles < sms ? (tiles > 0 ? tiles : 1) : sms);
}

// Adjoint of the BF16 network: head on CUDA cores, hidden layers top down on
// tcgen05; per-CTA weight-gradient partials [n_cta][n_params] for the caller
// to reduce.
geraf_status mlp_tc_backward_impl(const geraf_field_desc* d, const float* xyz, int64_t n, const void* saved,
                                  const float* d_sdf, const float* d_grad, const float* d_refl, float* zbar,
                                  float* partial, int64_t n_params, int n_cta, cudaStream_t st) {
    TcGeom g;
    if (!make_tc_geom(d, n, &g)) return GERAF_ERR_UNSUPPORTED;
    {
        const geraf_status as = smem_attrs(227 * 1024, "shared-memory opt-in", mlp_tc_layer_bwd_kernel);
        if (as != GERAF_OK) return as;
    }
    TcBwdArgs a{g, d->params, xyz, static_cast<const float*>(saved), d_sdf, d_grad, d_refl, zbar, partial,
                n_params, 0, device_error_word()};
    mlp_tc_head_bwd_kernel<<<n_cta, HB_THREADS, 0, st>>>(a);
    for (int l = g.NH - 1; l >= 0; --l) {
        a.layer = l;
        const size_t smem = bwd_layout(l == 0 ? g.K0p : TW).total + 1024;
        mlp_tc_layer_bwd_kernel<<<n_cta, BTHREADS, smem, st>>>(a);
    }
    return cuda_status(cudaGetLastError(), "fields_backward(mlp bf16)");
}

}  // namespace geraf
