// The paper's field networks (App. C "Training Setup": an SDF network of 8
// softplus layers of 256 on a 10-octave positional encoding and a separate
// reflectivity network of 4 layers of 256 on the same encoding; section 5.2
// "Signal representation"), and any other layer-by-layer network of width
// 64 .. 256 (a multiple of 64), in BF16 on the fifth-generation tensor cores
// with FP32 accumulation: the BF16 network reading (weights and every hidden
// layer's inputs rounded to bfloat16, bias, nonlinearity and head in FP32,
// straight-through adjoint).
//
// Every contraction is one generic tcgen05 GEMM, D[128 x N] = sum over K of
// A[128 x K] B[N x K]^T, N <= 256, both operands BF16 in a tiled K-major
// layout in global memory that equals the no-swizzle canonical shared-memory
// layout: 128-row x 64-column blocks of 16 KB (8 x 16-byte core matrices per
// 8-row group, groups 1 KB apart), so that one 1-D bulk copy moves a block.
// Rows of the activations are r = j S + s (point j, stream s: the value and,
// for the SDF network, the three x-tangents, S = 4).
//   forward layer:  A = Z (layer input, rows x K_in), B = W (units x K_in);
//                   epilogue: bias, softplus / sigmoid(beta h0) dh, the FP32
//                   pre-activations H (kept for the adjoint), the BF16 output
//                   Z' and its transpose Z'^T (the weight gradient's operand);
//   input adjoint:  A = Hb (rows x units, hi and lo BF16 parts), B = W^T;
//   weight gradient: A = Hb^T (units x rows), B = Z^T (K_in x rows), summed
//                   over a split of the rows in TMEM, partials in FP64 later.
// CTA: warp 0 issues the bulk copies into a ring of stages, one thread of
// warp 1 issues the MMAs (accumulator in TMEM), then all four warps read
// their 32 TMEM lanes for the epilogue. Every wait is bounded.
#include <cuda_bf16.h>
#include <math.h>

#include <algorithm>

#include "tcgen05.cuh"

namespace geraf {

namespace {

constexpr int WB = 128;                  // rows of a tile block (MMA M)
constexpr int WC = 64;                   // columns (K) of a tile block
constexpr uint32_t BLK = WB * WC * 2;    // bytes of a tile block: 16 KB
constexpr uint32_t W_LBO = 128;          // K-direction core-matrix stride
constexpr uint32_t W_SBO = 1024;         // 8-row group stride inside a block
constexpr int WT = 128;                  // threads per CTA
constexpr int WNH = 16;                  // hidden layers of one network

// byte offset of element (r, k) in a tiled [rows][cols] BF16 matrix with kc
// column blocks per row block
__host__ __device__ __forceinline__ size_t tiled_off(int64_t r, int64_t k, int64_t kc) {
    return ((size_t)(r / WB) * kc + (size_t)(k / WC)) * BLK + (size_t)((r % WB) >> 3) * W_SBO +
           (size_t)((k % WC) >> 3) * W_LBO + (size_t)(r & 7) * 16u + (size_t)(k & 7) * 2u;
}

struct TNet {
    const float* params;          // this network's packed FP32 parameters
    int L, K0, K0p, W, NH, S, head_out;
    float beta, inv_beta, cx, cy, cz, half;
    int64_t off_w[WNH + 1], off_b[WNH + 1];
    int64_t n_params;
    int k_in(int l) const { return l == 0 ? K0 : W; }
    int k_pad(int l) const { return l == 0 ? K0p : W; }
};

// softplus_beta(h) and sigmoid(beta h) from one exponential e = exp(-beta |h|);
// every kernel of this file that forms an activation calls this function, so
// the adjoint's BF16 operands are bit for bit those of the forward
__device__ __forceinline__ void wact(float h, float beta, float inv_beta, float& sp, float& sg) {
    const float e = __expf(-beta * fabsf(h));
    const float r = __fdividef(1.0f, 1.0f + e);
    sg = h >= 0.0f ? r : e * r;
    sp = fmaf(log1pf(e), inv_beta, fmaxf(h, 0.0f));
}
__device__ __forceinline__ float bfr(float v) { return __bfloat162float(__float2bfloat16_rn(v)); }
__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    return (uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(lo)) |
           ((uint32_t)__bfloat16_as_ushort(__float2bfloat16_rn(hi)) << 16);
}

// 8x8 transpose of 16-bit values across each aligned group of 8 lanes: lane i
// holds row i (p[k] = elements 2k, 2k + 1) on entry and column i on exit
__device__ __forceinline__ void tr8x8(uint32_t (&p)[4]) {
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

// 16 bytes (8 BF16 values of one row, columns k0 .. k0 + 7) at (r, k0) of a
// tiled matrix, and the same 8 columns of the 8 rows r0 .. r0 + 7 of this
// lane's group written transposed, as 16 bytes at (k0 + i, r0) of the
// transposed tiled matrix (lane i of the group); rows past `valid` as zeros
__device__ __forceinline__ void put_row8(unsigned char* __restrict__ z, int64_t z_kc, unsigned char* __restrict__ zt,
                                         int64_t zt_kc, int64_t r, int k0, const float (&v)[8], bool valid) {
    uint32_t q[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) q[k] = valid ? pack2(v[2 * k], v[2 * k + 1]) : 0u;
    if (z) *reinterpret_cast<uint4*>(z + tiled_off(r, k0, z_kc)) = make_uint4(q[0], q[1], q[2], q[3]);
    if (zt) {
        tr8x8(q);
        const int64_t r0 = r & ~(int64_t)7;
        *reinterpret_cast<uint4*>(zt + tiled_off(k0 + (threadIdx.x & 7), r0, zt_kc)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
}

// ------------------------------------------------------------- encoding
// Row r = j S + s of the positional encoding (section 9.3) of point j, BF16:
// Z0 [R][K0p] and Z0^T [K0p][R], tiled. Thread = row, 128 threads per block
// and R a multiple of 128, so every lane of a warp is in range (the
// transposed stores pair each aligned group of 8 rows).
__global__ void __launch_bounds__(128) wtc_encode_kernel(const float* __restrict__ xyz, int64_t n, TNet g,
                                                         int64_t R, unsigned char* __restrict__ z,
                                                         unsigned char* __restrict__ zt) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const bool valid = r < n * g.S;
    const int64_t j = valid ? r / g.S : 0;
    const int s = valid ? (int)(r % g.S) : 0;
    const int64_t z_kc = g.K0p / WC, zt_kc = R / WC;
    // the encoded coordinate of each axis, once per row (FP64: the divide is the
    // expensive part on this GPU's FP64 pipe)
    double xt[3];
    const double pih = 3.14159265358979323846 / (double)g.half;   // 2^k pi / half = 2^k (pi / half) exactly
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float x = xyz[(int64_t)d * n + j];
        const float c = d == 0 ? g.cx : (d == 1 ? g.cy : g.cz);
        xt[d] = ((double)x - (double)c) / (double)g.half;
    }
    for (int k0 = 0; k0 < g.K0p; k0 += 8) {
        float v[8];
#pragma unroll
        for (int e = 0; e < 8; ++e) {
            const int f = k0 + e;
            float val = 0.0f;
            const int k = f / 6, rem = f % 6, d = rem % 3;
            if (valid && f < g.K0 && (s == 0 || s - 1 == d)) {   // a tangent row is zero off its own axis
                const bool is_cos = rem >= 3;
                const double t2 = xt[d] * (double)(1 << k);
                const double rr = t2 - 2.0 * rint(0.5 * t2);          // exact reduction mod 2
                float sn, cs;
                sincospif((float)rr, &sn, &cs);                       // sin, cos of 2^k pi xt
                if (s == 0) {
                    val = is_cos ? cs : sn;
                } else if (s - 1 == d) {
                    const float wk = (float)((double)(1 << k) * pih);
                    val = is_cos ? -wk * sn : wk * cs;
                }
            }
            v[e] = val;
        }
        put_row8(z, z_kc, zt, zt_kc, r, k0, v, valid);
    }
}

// ------------------------------------------------------------ weights
// Layer weights W [out][in] (FP32, packed parameters) as BF16 tiled operands:
// wt = W [out][in_pad] (the forward's B), wtt = W^T [in_pad][out] (the input
// adjoint's B); columns in .. in_pad - 1 zero. Thread = (unit, 8 columns).
__global__ void wtc_prep_weights(const float* __restrict__ W, int out, int in, int in_pad,
                                 unsigned char* __restrict__ wt, unsigned char* __restrict__ wtt) {
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int groups = in_pad / 8;
    if (idx >= (int64_t)out * groups) return;
    const int u = (int)(idx / groups), k0 = (int)(idx % groups) * 8;
    float v[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) v[e] = k0 + e < in ? W[(int64_t)u * in + k0 + e] : 0.0f;
    if (wt) {
        uint32_t q[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) q[k] = pack2(v[2 * k], v[2 * k + 1]);
        *reinterpret_cast<uint4*>(wt + tiled_off(u, k0, in_pad / WC)) = make_uint4(q[0], q[1], q[2], q[3]);
    }
    if (wtt)
#pragma unroll
        for (int e = 0; e < 8; ++e)
            *reinterpret_cast<__nv_bfloat16*>(wtt + tiled_off(k0 + e, u, out / WC)) = __float2bfloat16_rn(v[e]);
}

// --------------------------------------------------------------- GEMM
enum { WTC_FWD = 0, WTC_DZ = 1, WTC_DW = 2 };
constexpr int WST_MAX = 4;

struct WtcArgs {
    int mode;
    const unsigned char* a0;   // A (or its hi part), tiled
    const unsigned char* a1;   // A's lo part or null
    int64_t a_kc;              // column blocks per row block of A
    const unsigned char* b;    // B, tiled
    int64_t b_kc;
    int n;                     // N = rows of B used, a multiple of 16, <= 256
    int64_t k_chunks;          // 64-column chunks of the contraction
    int64_t chunks_per_cta;    // DW: chunks per split (grid.x = splits); else k_chunks
    int stages;                // ring stages (2 .. WST_MAX)
    // forward epilogue
    const float* bias;
    float beta, inv_beta;
    int S;
    int64_t rows_valid;        // FWD, DZ: rows with data; DW: A rows (units) with data
    float* out;                // FWD: H [rows][ld]; DZ: the input adjoint [rows][ld]
    int64_t ld;
    unsigned char* z;          // FWD: the BF16 activation, tiled [R][n]
    int64_t z_kc;
    unsigned char* zt;         // FWD: its transpose, tiled [n][R]
    int64_t zt_kc;
    int n_valid;               // DZ, DW: output columns written
    float* partial;            // DW: partial[split * p_stride + p_off + unit * n_valid + k]
    int64_t p_stride, p_off;
    int* err;
};

__host__ __device__ inline size_t wtc_stage_bytes(int nsrc, int n) {
    return ((size_t)nsrc * BLK + (size_t)n * 128 + 1023) & ~(size_t)1023;
}
size_t wtc_smem(int nsrc, int n, int stages) { return 1024 + (size_t)stages * wtc_stage_bytes(nsrc, n) + 128; }

__global__ void __launch_bounds__(WT, 1) wtc_gemm_kernel(const WtcArgs a) {
    extern __shared__ __align__(1024) unsigned char wsm_raw[];
    unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(wsm_raw) + 1023) & ~(uintptr_t)1023);
    const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
    const int nsrc = a.a1 ? 2 : 1;
    const uint32_t stage_bytes = (uint32_t)wtc_stage_bytes(nsrc, a.n);
    unsigned char* bars = sm + (size_t)a.stages * stage_bytes;
    uint64_t* full = reinterpret_cast<uint64_t*>(bars);                 // [WST_MAX]
    uint64_t* empty = full + WST_MAX;                                   // [WST_MAX]
    uint64_t* done = empty + WST_MAX;
    uint32_t* tslot = reinterpret_cast<uint32_t*>(done + 1);
    int* abort_flag = reinterpret_cast<int*>(tslot + 1);
    int* issued = abort_flag + 1;
    const int64_t mb = a.mode == WTC_DW ? blockIdx.y : blockIdx.x;
    const int64_t c0 = a.mode == WTC_DW ? (int64_t)blockIdx.x * a.chunks_per_cta : 0;
    const int64_t c1 = a.mode == WTC_DW ? min(a.k_chunks, c0 + a.chunks_per_cta) : a.k_chunks;
    const int nk = (int)max((int64_t)0, c1 - c0);
    if (t == 0) {
        for (int s = 0; s < WST_MAX; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(done, 1);
        *abort_flag = 0;
        *issued = 0;
        fence_barrier_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 256);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tbase = *tslot;
    const uint32_t b_bytes = (uint32_t)a.n * 128u;

    if (warp == 0 && lane == 0) {
        // producer: stage s of chunk c holds A (hi, lo) then B's row blocks
        for (int c = 0; c < nk; ++c) {
            const int s = c % a.stages;
            if (c >= a.stages && !mbar_wait(&empty[s], ((c / a.stages) - 1) & 1)) {
                atomicOr(abort_flag, 1);
                break;
            }
            if (*(volatile int*)abort_flag) break;
            unsigned char* st = sm + (size_t)s * stage_bytes;
            mbar_arrive_expect_tx(&full[s], (uint32_t)nsrc * BLK + b_bytes);
            const int64_t kc = c0 + c;
            tma_load_1d(st, a.a0 + ((size_t)mb * a.a_kc + kc) * BLK, BLK, &full[s]);
            if (a.a1) tma_load_1d(st + BLK, a.a1 + ((size_t)mb * a.a_kc + kc) * BLK, BLK, &full[s]);
            for (int nb = 0; nb * WB < a.n; ++nb) {
                const uint32_t bytes = (uint32_t)min(WB, a.n - nb * WB) * 128u;
                tma_load_1d(st + (size_t)nsrc * BLK + (size_t)nb * BLK, a.b + ((size_t)nb * a.b_kc + kc) * BLK, bytes,
                            &full[s]);
            }
            *(volatile int*)issued = c + 1;
        }
    } else if (warp == 1 && lane == 0) {
        // MMA issuer: D[128][n] (+)= A B^T, K = 16 per instruction
        const uint32_t idesc = tc::idesc_bf16(128, a.n);
        for (int c = 0; c < nk; ++c) {
            const int s = c % a.stages;
            if (!mbar_wait(&full[s], (c / a.stages) & 1)) {
                atomicOr(abort_flag, 1);
                break;
            }
            tc::fence_after_sync();
            const uint32_t st = smem_u32(sm + (size_t)s * stage_bytes);
            const uint32_t bs = st + (uint32_t)nsrc * BLK;
            for (int src = 0; src < nsrc; ++src)
                for (int q = 0; q < WC / 16; ++q)
                    tc::mma_bf16(tbase, tc::smem_desc(st + (uint32_t)src * BLK + q * 256u, W_LBO, W_SBO),
                                 tc::smem_desc(bs + q * 256u, W_LBO, W_SBO), idesc,
                                 (c > 0 || src > 0 || q > 0) ? 1u : 0u);
            tc::mma_commit(&empty[s]);
        }
        tc::mma_commit(done);      // arrives once every MMA issued above has completed
    }
    // epilogue: warp w owns TMEM lanes 32 w .. 32 w + 31 (rows of the tile, or units for DW)
    const bool ok = mbar_wait(done, 0);
    if (!ok) atomicOr(abort_flag, 1);
    tc::fence_after_sync();
    __syncthreads();
    __syncwarp();
    if (!*abort_flag && nk > 0) {
        const int64_t row = mb * WB + warp * 32 + lane;
        const uint32_t taddr = tbase + ((uint32_t)(warp * 32) << 16);
        for (int u0 = 0; u0 < a.n; u0 += 32) {
            float acc[32];
            tc::tmem_ld32(taddr + (uint32_t)u0, acc);
            if (a.mode == WTC_FWD) {
                const int s = (int)(row % a.S);
                const bool valid = row < a.rows_valid;
#pragma unroll
                for (int i = 0; i < 32; ++i) acc[i] += s == 0 ? a.bias[u0 + i] : 0.0f;   // bias on value rows
                if (valid)
#pragma unroll
                    for (int i = 0; i < 32; i += 4)
                        *reinterpret_cast<float4*>(a.out + row * a.ld + u0 + i) =
                            make_float4(acc[i], acc[i + 1], acc[i + 2], acc[i + 3]);
#pragma unroll
                for (int g8 = 0; g8 < 4; ++g8) {
                    float v[8];
#pragma unroll
                    for (int e = 0; e < 8; ++e) {
                        const float h = acc[8 * g8 + e];
                        const float h0 = __shfl_sync(0xffffffffu, h, lane - s);
                        float sp, sg;
                        wact(h0, a.beta, a.inv_beta, sp, sg);
                        v[e] = s == 0 ? sp : sg * h;
                    }
                    put_row8(a.z, a.z_kc, a.zt, a.zt_kc, row, u0 + 8 * g8, v, valid);
                }
            } else {
                // the warp's 32 rows x 32 columns through a padded shared-memory
                // transpose (the stage ring, free once every MMA has completed),
                // so that each store writes 32 consecutive columns of one row
                float* tb = reinterpret_cast<float*>(sm) + warp * 32 * 33;
#pragma unroll
                for (int i = 0; i < 32; ++i) tb[lane * 33 + i] = acc[i];
                __syncwarp();
                const int64_t row0 = mb * WB + warp * 32;
                const bool col_ok = u0 + lane < a.n_valid;
                for (int i = 0; i < 32; ++i) {
                    const int64_t r = row0 + i;
                    if (r < a.rows_valid && col_ok) {
                        const float v = tb[i * 33 + lane];
                        if (a.mode == WTC_DZ)
                            a.out[r * a.ld + u0 + lane] = v;
                        else
                            a.partial[(size_t)blockIdx.x * a.p_stride + a.p_off + (size_t)r * a.n_valid + u0 + lane] = v;
                    }
                }
                __syncwarp();
            }
        }
    }
    if (*abort_flag && t == 0) {
        atomicOr(a.err, 1);
        // bounded: let the copies still in flight land before the shared memory is handed on
        const int n_issued = *(volatile int*)issued;
        for (int c = max(0, n_issued - a.stages); c < n_issued; ++c)
            mbar_wait(&full[c % a.stages], (c / a.stages) & 1, 100000000ull);
        if (!ok) mbar_wait(done, 0, 100000000ull);
    }
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    if (warp == 0) tc::tmem_dealloc(tbase, 256);
}

// ------------------------------------------------- pre-activation adjoint
// Hb from the activation adjoint zbar and the pre-activations H (FP32,
// [rows][W]): hb0 = zb0 sg + (sum_s zb_s h_s) beta sg (1 - sg) on value rows,
// hb_s = sg zb_s on tangent rows, sg = sigmoid(beta h0) of the point's value
// row. Written as BF16 hi + lo parts, each tiled twice: [R][W] (the input
// adjoint's A) and [W][R] (the weight gradient's A); rows past the data are
// zeros. Value-row sums per 64-row block go to bsum [R/64][W].
// Block = 8 warps x 8 rows (64 rows) x 32 units; lane = (row & 7, 8-unit group).
__global__ void __launch_bounds__(256) wtc_hbar_kernel(const float* __restrict__ zbar, const float* __restrict__ H,
                                                       int W, int S, float beta, float inv_beta, int64_t rows_valid,
                                                       int64_t R, unsigned char* __restrict__ hb_hi,
                                                       unsigned char* __restrict__ hb_lo,
                                                       unsigned char* __restrict__ hbt_hi,
                                                       unsigned char* __restrict__ hbt_lo, float* __restrict__ bsum) {
    __shared__ float red[8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t r = (int64_t)blockIdx.x * 64 + warp * 8 + (lane & 7);
    const int u0 = blockIdx.y * 32 + (lane >> 3) * 8;
    const bool valid = r < rows_valid;
    const int s = (int)(r % S);
    float zb[8], h[8];
    if (valid) {
        const float4* zp = reinterpret_cast<const float4*>(zbar + r * W + u0);
        const float4* hp = reinterpret_cast<const float4*>(H + r * W + u0);
        const float4 z0 = zp[0], z1 = zp[1], h0v = hp[0], h1v = hp[1];
        zb[0] = z0.x; zb[1] = z0.y; zb[2] = z0.z; zb[3] = z0.w; zb[4] = z1.x; zb[5] = z1.y; zb[6] = z1.z; zb[7] = z1.w;
        h[0] = h0v.x; h[1] = h0v.y; h[2] = h0v.z; h[3] = h0v.w; h[4] = h1v.x; h[5] = h1v.y; h[6] = h1v.z; h[7] = h1v.w;
    } else {
#pragma unroll
        for (int e = 0; e < 8; ++e) zb[e] = h[e] = 0.0f;
    }
    float hb[8], hl[8], bs[8];
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        const float h0 = __shfl_sync(0xffffffffu, h[e], lane - s);
        float sp, sg;
        wact(h0, beta, inv_beta, sp, sg);
        float v;
        if (S == 4) {
            float t = s != 0 ? zb[e] * h[e] : 0.0f;          // the point's three tangent rows
            t += __shfl_xor_sync(0xffffffffu, t, 1);
            t += __shfl_xor_sync(0xffffffffu, t, 2);
            v = s == 0 ? fmaf(t, beta * sg * (1.0f - sg), zb[e] * sg) : sg * zb[e];
        } else {
            v = zb[e] * sg;
        }
        v = valid ? v : 0.0f;
        hb[e] = bfr(v);
        hl[e] = v - hb[e];
        bs[e] = s == 0 ? v : 0.0f;
    }
    put_row8(hb_hi, W / WC, hbt_hi, R / WC, r, u0, hb, true);
    put_row8(hb_lo, W / WC, hbt_lo, R / WC, r, u0, hl, true);
    // bias sums: the warp's 8 rows (lanes with the same unit group), then the 8 warps in order
#pragma unroll
    for (int e = 0; e < 8; ++e) {
        float v = bs[e];
        v += __shfl_xor_sync(0xffffffffu, v, 1);
        v += __shfl_xor_sync(0xffffffffu, v, 2);
        v += __shfl_xor_sync(0xffffffffu, v, 4);
        if ((lane & 7) == 0) red[warp][(lane >> 3) * 8 + e] = v;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        float v = 0.0f;
        for (int w = 0; w < 8; ++w) v += red[w][threadIdx.x];
        bsum[(size_t)blockIdx.x * W + blockIdx.y * 32 + threadIdx.x] = v;
    }
}

// bias gradient of a layer: the 64-row block sums. Block = 32 units x
// BR_SLICES slices of the row blocks; each thread sums its slice in block
// order with Kahan compensation in FP32 (FP64 is a small fraction of FP32 on
// this part), the slices are added in slice order in FP64, so the result does
// not depend on the launch.
constexpr int BR_SLICES = 32;
__global__ void __launch_bounds__(32 * BR_SLICES) wtc_bias_reduce(const float* __restrict__ bsum, int64_t n_blocks,
                                                                  int W, float* __restrict__ out) {
    __shared__ double part[BR_SLICES][32];
    const int lu = threadIdx.x & 31, sl = threadIdx.x >> 5;
    const int u = blockIdx.x * 32 + lu;
    const int64_t per = (n_blocks + BR_SLICES - 1) / BR_SLICES;
    const int64_t b0 = sl * per, b1 = min(n_blocks, b0 + per);
    float acc = 0.0f, cmp = 0.0f;
    if (u < W)
        for (int64_t b = b0; b < b1; ++b) {
            const float y = bsum[(size_t)b * W + u] - cmp;
            const float t = acc + y;
            cmp = (t - acc) - y;
            acc = t;
        }
    part[sl][lu] = (double)acc - (double)cmp;
    __syncthreads();
    if (sl == 0 && u < W) {
        double s = 0.0;
        for (int q = 0; q < BR_SLICES; ++q) s += part[q][lu];
        out[u] = (float)s;
    }
}

// ------------------------------------------------------------------ head
// One warp per point: the head on the last hidden layer's BF16 activations,
// formed from the saved pre-activations exactly as the GEMM epilogue formed
// them. out_f / out_grad: head row 0; a from row a_row (1: shared trunk,
// 0: reflectivity network, -1: none).
__global__ void wtc_head_fwd_kernel(TNet g, int64_t n, const float* __restrict__ H, float* __restrict__ out_f,
                                    float* __restrict__ out_grad, float* __restrict__ out_a,
                                    float* __restrict__ a_saved, int a_row) {
    const int64_t j = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (j >= n) return;
    const float* Wh = g.params + g.off_w[g.NH];
    const float* bh = g.params + g.off_b[g.NH];
    const float* h0 = H + (j * g.S) * g.W;
    float acc[5] = {0.0f, 0.0f, 0.0f, 0.0f, 0.0f};
    for (int u = lane; u < g.W; u += 32) {
        const float hv = h0[u];
        float sp, sg;
        wact(hv, g.beta, g.inv_beta, sp, sg);
        const float z0 = bfr(sp);
        acc[0] = fmaf(Wh[u], z0, acc[0]);
        if (a_row > 0) acc[4] = fmaf(Wh[(int64_t)a_row * g.W + u], z0, acc[4]);
        if (g.S == 4 && out_grad)
#pragma unroll
            for (int s = 1; s < 4; ++s) acc[s] = fmaf(Wh[u], bfr(sg * h0[(int64_t)s * g.W + u]), acc[s]);
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
            const float x = a_row == 0 ? acc[0] + bh[0] : acc[4] + bh[a_row];
            const float a = 1.0f / (1.0f + expf(-x));
            if (out_a) out_a[j] = a;
            if (a_saved) a_saved[j] = a;
        }
    }
}

// Head adjoint: block (split, 32-unit chunk), threadIdx.x = unit, threadIdx.y
// = one of 8 point lanes over the split's points. Writes the top activation
// adjoint zbar[(j S + s) W + u] (through the FP32 head weights) and the head's
// gradient partials from the BF16 activations the forward multiplied.
__global__ void __launch_bounds__(256) wtc_head_bwd_kernel(TNet g, int64_t n, int64_t pps,
                                                           const float* __restrict__ H,
                                                           const float* __restrict__ a_saved,
                                                           const float* __restrict__ d_f,
                                                           const float* __restrict__ d_grad,
                                                           const float* __restrict__ d_a, int refl_net,
                                                           float* __restrict__ zbar, float* __restrict__ partial,
                                                           int64_t split_stride) {
    __shared__ float red[4][8][32];
    const int sp_ = blockIdx.x;
    const int u = blockIdx.y * 32 + threadIdx.x;
    const int64_t j0 = (int64_t)sp_ * pps, j1 = min(n, j0 + pps);
    const float* Wh = g.params + g.off_w[g.NH];
    float gw0 = 0.0f, gw1 = 0.0f, gb0 = 0.0f, gb1 = 0.0f;
    if (u < g.W) {
        const float w0 = Wh[u], w1 = g.head_out == 2 ? Wh[g.W + u] : 0.0f;
        for (int64_t j = j0 + threadIdx.y; j < j1; j += 8) {
            const float* h = H + (j * g.S) * g.W;
            const float hv = h[u];
            float spv, sg;
            wact(hv, g.beta, g.inv_beta, spv, sg);
            const float z0 = bfr(spv);
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
#pragma unroll
                for (int s = 1; s < 4; ++s) {
                    const float dg = d_grad ? d_grad[(int64_t)(s - 1) * n + j] : 0.0f;
                    zb[(int64_t)s * g.W + u] = w0 * dg;
                    gw0 = fmaf(dg, bfr(sg * h[(int64_t)s * g.W + u]), gw0);
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
        float* part = partial + (int64_t)sp_ * split_stride;
        part[g.off_w[g.NH] + u] = t0;
        if (g.head_out == 2) part[g.off_w[g.NH] + g.W + u] = t1;
        if (u == 0) {
            part[g.off_b[g.NH]] = b0;
            if (g.head_out == 2) part[g.off_b[g.NH] + 1] = b1;
        }
    }
}

// the per-split parameter-gradient partials summed in split order, Kahan
// compensated in FP32 (deterministic; FP64 is a small fraction of FP32 here)
__global__ void wtc_reduce_partials(const float* __restrict__ partial, int n_split, int64_t stride, int64_t n,
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

inline unsigned tdiv(int64_t a, int64_t b) { return (unsigned)((a + b - 1) / b); }
inline int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

bool make_tnet(const float* params, int L, int W, int NH, int head_out, int S, const geraf_field_desc* d, TNet* g) {
    if (L < 1 || L > 21 || W < 64 || W > 256 || (W % 64) != 0 || NH < 1 || NH > WNH || !(d->half > 0.0f)) {
        set_error("fields(bf16): layer-by-layer BF16 networks need 1 <= n_levels <= 21, a width that is a multiple "
                  "of 64 in [64, 256], 1 <= hidden layers <= %d and half > 0", WNH);
        return false;
    }
    g->params = params;
    g->L = L;
    g->K0 = 6 * L;
    g->K0p = (int)round_up(g->K0, WC);
    if (g->K0p > 256) {
        set_error("fields(bf16): encoding wider than 256 features");
        return false;
    }
    g->W = W;
    g->NH = NH;
    g->S = S;
    g->head_out = head_out;
    g->beta = d->beta;
    g->inv_beta = 1.0f / d->beta;
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
    return true;
}

struct TNets {
    TNet sdf, refl;
    int two;
    int64_t n_params;
};

bool make_tnets(const geraf_field_desc* d, int S_sdf, TNets* nets) {
    nets->two = d->refl_hidden > 0;
    if (!make_tnet(d->params, d->n_levels, d->width, d->n_hidden, nets->two ? 1 : 2, S_sdf, d, &nets->sdf))
        return false;
    nets->n_params = nets->sdf.n_params;
    if (nets->two) {
        if (!make_tnet(d->params + nets->sdf.n_params, d->n_levels, d->refl_width, d->refl_hidden, 1, 1, d,
                       &nets->refl))
            return false;
        nets->n_params += nets->refl.n_params;
    }
    return true;
}

// `saved` of one network at its full stream count (byte offsets from the
// network's base): per layer the BF16 weights (tiled), the BF16 transposed
// layer input Z^T (tiled) and the FP32 pre-activations H; two BF16 tiled
// activation buffers the forward alternates between.
struct TLayout {
    size_t wt[WNH], zt[WNH], H[WNH], zbuf[2];
    size_t bytes;
};
TLayout layout_of(const TNet& g, int64_t n) {
    TLayout L{};
    const int64_t R = round_up(n * g.S, WB);
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = align_up(off, 256);
        off = o + bytes;
        return o;
    };
    for (int l = 0; l < g.NH; ++l) L.wt[l] = take((size_t)round_up(g.W, WB) * g.k_pad(l) * 2);
    for (int l = 0; l < g.NH; ++l) L.zt[l] = take((size_t)round_up(g.k_pad(l), WB) * R * 2);
    for (int l = 0; l < g.NH; ++l) L.H[l] = take((size_t)n * g.S * g.W * sizeof(float));
    for (int b = 0; b < 2; ++b) L.zbuf[b] = take((size_t)R * std::max(g.K0p, g.W) * 2);
    L.bytes = align_up(off, 256);
    return L;
}

WtcArgs gemm_args(int mode, int* err) {
    WtcArgs a{};
    a.mode = mode;
    a.stages = 2;
    a.S = 1;
    a.err = err;
    return a;
}

geraf_status launch_gemm(const WtcArgs& a, dim3 grid, cudaStream_t st) {
    const size_t smem = wtc_smem(a.a1 ? 2 : 1, a.n, a.stages);
    wtc_gemm_kernel<<<grid, WT, smem, st>>>(a);
    return cuda_status(cudaGetLastError(), "fields(bf16 layers): gemm");
}

// forward of one network: weights to BF16 tiles, encoding, the hidden layers
// (GEMM + fused activation epilogue), then the head from the last layer's H
geraf_status tnet_forward(const TNet& g, const float* xyz, int64_t n, unsigned char* base, const TLayout& L,
                          float* out_f, float* out_grad, float* out_a, float* a_saved, int a_row, cudaStream_t st) {
    const int64_t rows = n * g.S, R = round_up(rows, WB);
    int* err = device_error_word();
    for (int l = 0; l < g.NH; ++l)
        wtc_prep_weights<<<tdiv((int64_t)g.W * (g.k_pad(l) / 8), 256), 256, 0, st>>>(
            g.params + g.off_w[l], g.W, g.k_in(l), g.k_pad(l), base + L.wt[l], nullptr);
    wtc_encode_kernel<<<(unsigned)(R / WB), WB, 0, st>>>(xyz, n, g, R, base + L.zbuf[0], base + L.zt[0]);
    for (int l = 0; l < g.NH; ++l) {
        const bool last = l + 1 == g.NH;
        WtcArgs a = gemm_args(WTC_FWD, err);
        a.a0 = base + L.zbuf[l & 1];
        a.a_kc = g.k_pad(l) / WC;
        a.b = base + L.wt[l];
        a.b_kc = g.k_pad(l) / WC;
        a.n = g.W;
        a.k_chunks = a.chunks_per_cta = g.k_pad(l) / WC;
        a.bias = g.params + g.off_b[l];
        a.beta = g.beta;
        a.inv_beta = g.inv_beta;
        a.S = g.S;
        a.rows_valid = rows;
        a.out = reinterpret_cast<float*>(base + L.H[l]);
        a.ld = g.W;
        a.z = last ? nullptr : base + L.zbuf[(l + 1) & 1];
        a.z_kc = g.W / WC;
        a.zt = last ? nullptr : base + L.zt[l + 1];
        a.zt_kc = R / WC;
        const geraf_status s = launch_gemm(a, dim3((unsigned)(R / WB)), st);
        if (s != GERAF_OK) return s;
    }
    const float* Hl = reinterpret_cast<const float*>(base + L.H[g.NH - 1]);
    wtc_head_fwd_kernel<<<tdiv(n * 32, 256), 256, 0, st>>>(g, n, Hl, out_f, out_grad, out_a, a_saved, a_row);
    return cuda_status(cudaGetLastError(), "fields(bf16 layers)");
}

struct TBwdWs {
    float *zA, *zB, *bsum, *partial;
    unsigned char *hb_hi, *hb_lo, *hbt_hi, *hbt_lo, *wtt;
};

// adjoint of one network: head, then per layer (top down) the pre-activation
// adjoint, the weight gradient over splits of the rows, and (above the first
// layer) the input adjoint
geraf_status tnet_backward(const TNet& g, int64_t n, const unsigned char* base, const TLayout& L,
                           const float* a_saved, const float* d_f, const float* d_grad, const float* d_a, int refl_net,
                           const TBwdWs& w, float* partial, int64_t stride, int splits, cudaStream_t st) {
    const int64_t rows = n * g.S, R = round_up(rows, WB);
    int* err = device_error_word();
    float* zA = w.zA;
    float* zB = w.zB;
    const int64_t pps = (n + splits - 1) / splits;
    wtc_head_bwd_kernel<<<dim3(splits, tdiv(g.W, 32)), dim3(32, 8), 0, st>>>(
        g, n, pps, reinterpret_cast<const float*>(base + L.H[g.NH - 1]), a_saved, d_f, d_grad, d_a, refl_net, zA,
        partial, stride);
    const int64_t k_chunks = R / WC;
    const int64_t cpc = (k_chunks + splits - 1) / splits;
    const unsigned dw_splits = (unsigned)((k_chunks + cpc - 1) / cpc);
    for (int l = g.NH - 1; l >= 0; --l) {
        const float* Hl = reinterpret_cast<const float*>(base + L.H[l]);
        wtc_hbar_kernel<<<dim3((unsigned)(R / 64), g.W / 32), 256, 0, st>>>(
            zA, Hl, g.W, g.S, g.beta, g.inv_beta, rows, R, w.hb_hi, w.hb_lo, w.hbt_hi, w.hbt_lo, w.bsum);
        wtc_bias_reduce<<<tdiv(g.W, 32), 32 * BR_SLICES, 0, st>>>(w.bsum, R / 64, g.W, partial + g.off_b[l]);
        WtcArgs a = gemm_args(WTC_DW, err);
        a.a0 = w.hbt_hi;
        a.a1 = w.hbt_lo;
        a.a_kc = R / WC;
        a.b = base + L.zt[l];
        a.b_kc = R / WC;
        a.n = g.k_pad(l);
        a.k_chunks = k_chunks;
        a.chunks_per_cta = cpc;
        a.rows_valid = g.W;
        a.n_valid = g.k_in(l);
        a.partial = partial;
        a.p_stride = stride;
        a.p_off = g.off_w[l];
        geraf_status s = launch_gemm(a, dim3(dw_splits, tdiv(g.W, WB)), st);
        if (s != GERAF_OK) return s;
        if (l > 0) {
            wtc_prep_weights<<<tdiv((int64_t)g.W * (g.W / 8), 256), 256, 0, st>>>(g.params + g.off_w[l], g.W, g.W,
                                                                                 g.W, nullptr, w.wtt);
            WtcArgs z = gemm_args(WTC_DZ, err);
            z.a0 = w.hb_hi;
            z.a1 = w.hb_lo;
            z.a_kc = g.W / WC;
            z.b = w.wtt;
            z.b_kc = g.W / WC;
            z.n = g.W;
            z.k_chunks = z.chunks_per_cta = g.W / WC;
            z.rows_valid = rows;
            z.out = zB;
            z.ld = g.W;
            z.n_valid = g.W;
            s = launch_gemm(z, dim3((unsigned)(R / WB)), st);
            if (s != GERAF_OK) return s;
            float* t = zA; zA = zB; zB = t;
        }
    }
    return cuda_status(cudaGetLastError(), "fields_backward(bf16 layers)");
}

int tc_splits(int64_t rows) {
    const int64_t chunks = round_up(rows, WB) / WC;
    return (int)std::max<int64_t>(1, std::min<int64_t>(device_sm_count() / 2, chunks));
}

}  // namespace

// ------------------------------------------------------------- entry glue
geraf_status mlp_wide_tc_saved_bytes(const geraf_field_desc* d, int64_t n, size_t* bytes) {
    TNets nets;
    if (!make_tnets(d, 4, &nets)) return GERAF_ERR_UNSUPPORTED;
    size_t b = layout_of(nets.sdf, n).bytes;
    if (nets.two) b += layout_of(nets.refl, n).bytes;
    *bytes = b + align_up((size_t)n * sizeof(float), 256);
    return GERAF_OK;
}

geraf_status mlp_wide_tc_forward(const geraf_field_desc* d, const float* xyz, int64_t n, float* sdf, float* grad,
                                 float* refl, void* saved, size_t saved_bytes, cudaStream_t st) {
    size_t need = 0;
    geraf_status s0 = mlp_wide_tc_saved_bytes(d, n, &need);
    if (s0 != GERAF_OK) return s0;
    if (!saved)
        return fail(GERAF_ERR_INVALID_ARG, "fields: this network keeps its layer activations in `saved`, which "
                                           "must be given even without a backward pass");
    if (saved_bytes < need) return fail(GERAF_ERR_WORKSPACE, "fields: saved %zu < %zu bytes", saved_bytes, need);
    TNets full, nets;
    make_tnets(d, 4, &full);
    if (!make_tnets(d, grad ? 4 : 1, &nets)) return GERAF_ERR_UNSUPPORTED;
    {
        const geraf_status as = smem_attrs((int)wtc_smem(2, 256, 2), "shared-memory opt-in", wtc_gemm_kernel);
        if (as != GERAF_OK) return as;
    }
    unsigned char* base = static_cast<unsigned char*>(saved);
    const TLayout Ls = layout_of(full.sdf, n);
    unsigned char* base_r = base + Ls.bytes;
    const TLayout Lr = nets.two ? layout_of(full.refl, n) : TLayout{};
    float* a_saved = reinterpret_cast<float*>(base_r + (nets.two ? Lr.bytes : 0));
    geraf_status s = tnet_forward(nets.sdf, xyz, n, base, Ls, sdf, grad, nets.two ? nullptr : refl,
                                  nets.two ? nullptr : a_saved, nets.two ? -1 : 1, st);
    if (s != GERAF_OK || !nets.two || !refl) return s;
    return tnet_forward(nets.refl, xyz, n, base_r, Lr, nullptr, nullptr, refl, a_saved, 0, st);
}

geraf_status mlp_wide_tc_backward(const geraf_field_desc* d, const float* xyz, int64_t n, const void* saved,
                                  const float* d_sdf, const float* d_grad, const float* d_refl, float* d_params,
                                  void* ws, size_t* ws_bytes, cudaStream_t st) {
    (void)xyz;
    TNets nets;
    if (!make_tnets(d, 4, &nets)) return GERAF_ERR_UNSUPPORTED;
    const int wmax = std::max(nets.sdf.W, nets.two ? nets.refl.W : 0);
    const int64_t rows = n * 4, R = round_up(rows, WB);
    const int splits = tc_splits(rows);
    WsCarver c(ws);
    TBwdWs w{};
    w.zA = c.take<float>((size_t)rows * wmax);
    w.zB = c.take<float>((size_t)rows * wmax);
    w.hb_hi = c.take<unsigned char>((size_t)R * wmax * 2);
    w.hb_lo = c.take<unsigned char>((size_t)R * wmax * 2);
    w.hbt_hi = c.take<unsigned char>((size_t)round_up(wmax, WB) * R * 2);
    w.hbt_lo = c.take<unsigned char>((size_t)round_up(wmax, WB) * R * 2);
    w.wtt = c.take<unsigned char>((size_t)round_up(wmax, WB) * wmax * 2);
    w.bsum = c.take<float>((size_t)(R / 64) * wmax);
    w.partial = c.take<float>((size_t)splits * nets.n_params);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used)
        return fail(GERAF_ERR_WORKSPACE, "fields_backward: workspace %zu < %zu bytes", *ws_bytes, c.used);
    if (!saved) return fail(GERAF_ERR_INVALID_ARG, "fields_backward: saved is NULL");
    {
        const geraf_status as = smem_attrs((int)wtc_smem(2, 256, 2), "shared-memory opt-in", wtc_gemm_kernel);
        if (as != GERAF_OK) return as;
    }
    // every split row of the partials not written below stays zero
    cudaError_t e = cudaMemsetAsync(w.partial, 0, (size_t)splits * nets.n_params * sizeof(float), st);
    if (e != cudaSuccess) return cuda_status(e, "fields_backward(bf16 layers) memset");
    const unsigned char* base = static_cast<const unsigned char*>(saved);
    const TLayout Ls = layout_of(nets.sdf, n);
    const unsigned char* base_r = base + Ls.bytes;
    const TLayout Lr = nets.two ? layout_of(nets.refl, n) : TLayout{};
    const float* a_saved = reinterpret_cast<const float*>(base_r + (nets.two ? Lr.bytes : 0));
    geraf_status s = tnet_backward(nets.sdf, n, base, Ls, a_saved, d_sdf, d_grad, nets.two ? nullptr : d_refl, 0, w,
                                   w.partial, nets.n_params, splits, st);
    if (s != GERAF_OK) return s;
    if (nets.two) {
        s = tnet_backward(nets.refl, n, base_r, Lr, a_saved, nullptr, nullptr, d_refl, 1, w,
                          w.partial + nets.sdf.n_params, nets.n_params, splits, st);
        if (s != GERAF_OK) return s;
    }
    wtc_reduce_partials<<<tdiv(nets.n_params, 256), 256, 0, st>>>(w.partial, splits, nets.n_params, nets.n_params,
                                                                   d_params);
    return cuda_status(cudaGetLastError(), "fields_backward(bf16 layers)");
}

}  // namespace geraf
