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

__device__ __forceinline__ float sp_b(float h, float beta) {
    return fmaxf(h, 0.0f) + log1pf(expf(-beta * fabsf(h))) / beta;
}
__device__ __forceinline__ float sgm(float x) { return 1.0f / (1.0f + expf(-x)); }

__device__ __forceinline__ void st_bf16(unsigned char* base, uint32_t off, float v) {
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
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

// shared memory: W tiles (BF16), X tile (BF16), biases and head (FP32), barrier, TMEM slot
__global__ void __launch_bounds__(TTHREADS, 1) mlp_tc_fwd_kernel(const TcFwdArgs a) {
    extern __shared__ __align__(1024) unsigned char smem[];
    const TcGeom& g = a.g;
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    // layout
    unsigned char* wt[4];
    uint32_t off = 0;
    for (int l = 0; l < g.NH; ++l) {
        wt[l] = smem + off;
        off += (uint32_t)TW * (l == 0 ? g.K0p : TW) * 2u;
    }
    off = (off + 1023u) & ~1023u;
    unsigned char* xt = smem + off;                        // [128 columns][128 K] BF16
    off += TCOL * TW * 2u;
    float* bias = reinterpret_cast<float*>(smem + off);    // [NH][128]
    off += g.NH * TW * 4u;
    float* head = reinterpret_cast<float*>(smem + off);    // W_f[128], W_a[128], b_f, b_a
    off += (2 * TW + 2) * 4u;
    off = (off + 7u) & ~7u;
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + off);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + off + 8);
    int* abort_flag = reinterpret_cast<int*>(smem + off + 12);

    // weights -> BF16 K-major tiles (encoding layer zero-padded to K0p)
    for (int l = 0; l < g.NH; ++l) {
        const int K = l == 0 ? g.K0 : TW, Kp = l == 0 ? g.K0p : TW;
        const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
        const float* W = a.params + g.off_w[l];
        for (int i = t; i < TW * Kp; i += TTHREADS) {
            const int u = i / Kp, k = i - u * Kp;
            st_bf16(wt[l], tc::kmajor_offset(u, k, TLBO, sbo), k < K ? W[u * K + k] : 0.0f);
        }
        for (int i = t; i < TW; i += TTHREADS) bias[l * TW + i] = a.params[g.off_b[l] + i];
    }
    for (int i = t; i < 2 * TW; i += TTHREADS) head[i] = a.params[g.off_w[g.NH] + i];
    if (t < 2) head[2 * TW + t] = a.params[g.off_b[g.NH] + t];
    if (t == 0) {
        mbar_init(bar, 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 128);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t idesc = tc::idesc_bf16(128, TCOL);
    uint32_t phase = 0;

    for (int tile = blockIdx.x; tile < g.n_tiles; tile += gridDim.x) {
        const int64_t j0 = (int64_t)tile * TTP;
        // positional encoding and its x-derivatives -> X (BF16, K = K0p)
        {
            const uint32_t sbo0 = (uint32_t)(g.K0p / 8) * 128u;
            for (int i = t; i < TCOL * (g.K0p - g.K0); i += TTHREADS) {
                const int c = i / (g.K0p - g.K0), k = g.K0 + i % (g.K0p - g.K0);
                st_bf16(xt, tc::kmajor_offset(c, k, TLBO, sbo0), 0.0f);
            }
            if (t < 3 * TTP) {
                const int p = t / 3, d = t - 3 * (t / 3);
                int64_t j = j0 + p;
                if (j >= g.n) j = g.n - 1;
                const float x = a.xyz[d * g.n + j];
                const float c = d == 0 ? g.cx : (d == 1 ? g.cy : g.cz);
                const double xt_ = ((double)x - (double)c) / (double)g.half;
                for (int k = 0; k < g.L; ++k) {
                    const double t2 = xt_ * (double)(1 << k);
                    const double r = t2 - 2.0 * rint(0.5 * t2);
                    float sn, cs;
                    sincospif((float)r, &sn, &cs);
                    const float wk = (float)((double)(1 << k) * 3.14159265358979323846 / (double)g.half);
                    const int fs = 6 * k + d, fc = 6 * k + 3 + d;
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        float vs, vc;
                        if (s == 0) { vs = sn; vc = cs; }
                        else if (s - 1 == d) { vs = wk * cs; vc = -wk * sn; }
                        else { vs = 0.0f; vc = 0.0f; }
                        st_bf16(xt, tc::kmajor_offset(4 * p + s, fs, TLBO, sbo0), vs);
                        st_bf16(xt, tc::kmajor_offset(4 * p + s, fc, TLBO, sbo0), vc);
                    }
                }
            }
        }
        for (int l = 0; l < g.NH; ++l) {
            const int Kp = l == 0 ? g.K0p : TW;
            const uint32_t sbo = (uint32_t)(Kp / 8) * 128u;
            tc::fence_async_smem();
            tc::fence_before_sync();
            __syncthreads();
            tc::fence_after_sync();
            if (t == 0) {
                const uint32_t wa = smem_u32(wt[l]), xa = smem_u32(xt);
                for (int s = 0; s < Kp / 16; ++s)
                    tc::mma_bf16(tbase, tc::smem_desc(wa + s * 256u, TLBO, sbo), tc::smem_desc(xa + s * 256u, TLBO, sbo),
                                 idesc, s > 0 ? 1u : 0u);
                tc::mma_commit(bar);
            }
            const bool ok = mbar_wait(bar, phase);
            phase ^= 1u;
            if (!ok) atomicOr(abort_flag, 1);
            tc::fence_after_sync();
            __syncthreads();
            if (*abort_flag) break;
            // epilogue: thread = unit u of TMEM lane u; 32 columns (8 points) per load
            const int u = warp * 32 + lane;
            const float bu = bias[l * TW + u];
            for (int cc = 0; cc < 4; ++cc) {
                float r[32];
                tc::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(cc * 32), r);
#pragma unroll
                for (int pp = 0; pp < 8; ++pp) {
                    const int p = cc * 8 + pp;
                    const float h = r[4 * pp] + bu;
                    const float sg = sgm(g.beta * h);
                    const float v[4] = {sp_b(h, g.beta), sg * r[4 * pp + 1], sg * r[4 * pp + 2], sg * r[4 * pp + 3]};
#pragma unroll
                    for (int s = 0; s < 4; ++s) st_bf16(xt, tc::kmajor_offset(4 * p + s, u, TLBO, 16u * 128u), v[s]);
                    const int64_t j = j0 + p;
                    if (a.saved && j < g.n) {
                        float* dst = a.saved + (((int64_t)l * g.n + j) * 4) * TW + u;
                        dst[0] = h;
                        dst[TW] = r[4 * pp + 1];
                        dst[2 * TW] = r[4 * pp + 2];
                        dst[3 * TW] = r[4 * pp + 3];
                    }
                }
            }
            tc::fence_before_sync();
        }
        if (*abort_flag) break;
        __syncthreads();
        // head from the last BF16 activations, thread = column
        {
            const int c = t, p = c >> 2, s = c & 3;
            const int64_t j = j0 + p;
            float v0 = 0.0f, v1 = 0.0f;
            for (int u8 = 0; u8 < TW; u8 += 8) {
                const uint4 raw = *reinterpret_cast<const uint4*>(xt + tc::kmajor_offset(c, u8, TLBO, 16u * 128u));
                const __nv_bfloat16* e = reinterpret_cast<const __nv_bfloat16*>(&raw);
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float x = __bfloat162float(e[q]);
                    v0 = fmaf(head[u8 + q], x, v0);
                    v1 = fmaf(head[TW + u8 + q], x, v1);
                }
            }
            if (j < g.n) {
                if (s == 0) {
                    a.sdf[j] = v0 + head[2 * TW];
                    const float av = sgm(v1 + head[2 * TW + 1]);
                    if (a.refl) a.refl[j] = av;
                    if (a.saved) a.saved[(int64_t)g.NH * g.n * 4 * TW + j] = av;
                } else if (a.grad) {
                    a.grad[(int64_t)(s - 1) * g.n + j] = v0;
                }
            }
        }
        __syncthreads();   // the next tile's encoding overwrites the tile the head read
    }
    if (*abort_flag && t == 0) {
        atomicOr(a.err, 1);
        mbar_wait(bar, phase ^ 1u, 100000000ull);   // bounded: let the timed-out MMA finish before TMEM is freed
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, 128);
}

size_t tc_fwd_smem(const TcGeom& g) {
    size_t off = 0;
    for (int l = 0; l < g.NH; ++l) off += (size_t)TW * (l == 0 ? g.K0p : TW) * 2;
    off = (off + 1023) & ~(size_t)1023;
    off += TCOL * TW * 2;
    off += g.NH * TW * 4 + (2 * TW + 2) * 4;
    off = (off + 7) & ~(size_t)7;
    return off + 16 + 1024;   // barrier, TMEM slot, abort flag; slack for the 1024-byte base alignment
}

}  // namespace

geraf_status mlp_tc_forward_impl(const geraf_field_desc* d, const float* xyz, int64_t n, float* sdf, float* grad,
                                 float* refl, void* saved, cudaStream_t st) {
    TcGeom g;
    if (!make_tc_geom(d, n, &g)) return GERAF_ERR_UNSUPPORTED;
    const size_t smem = tc_fwd_smem(g);
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(mlp_tc_fwd_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
        attr = true;
    }
    int n_cta = device_sm_count();
    if (n_cta > g.n_tiles) n_cta = g.n_tiles;
    TcFwdArgs a{g, d->params, xyz, sdf, grad, refl, static_cast<float*>(saved), device_error_word()};
    mlp_tc_fwd_kernel<<<n_cta, TTHREADS, smem, st>>>(a);
    return cuda_status(cudaGetLastError(), "fields(mlp bf16)");
}

}  // namespace geraf
