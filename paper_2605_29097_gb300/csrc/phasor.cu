// Phasor-sum kernels of the rendering path: signal tracing (render) and the
// matched filter (filter), each with its adjoint.
//
// Two kernel shapes cover the four sums:
//  * "to bins"  (render, filter backward): outputs indexed by (antenna, bin);
//    each thread owns one antenna x 32 consecutive bins, point tiles stream
//    through shared memory by TMA, the phasor steps across the 32 bins by the
//    angle-addition recurrence q <- q * exp(-j 2 pi df tau) from a fresh seed
//    exp(-j 2 pi f_32b tau), i.e. re-seeded every 32 bins. Per-pair quantities
//    (range as a double-single, amplitude, step phasor) are computed once per
//    (antenna, point) by the whole CTA and shared by the 32-bin blocks of that
//    antenna. Split over points; per-thread sums are two-level (FP32 inner
//    sum over 128 points, Kahan-compensated outer sum), split partials are
//    added in FP64 by a second kernel in a fixed order.
//  * "to points" (filter, render backward): outputs indexed by point/voxel;
//    each thread owns 2 points, antenna tiles (position + the 32-bin-padded
//    signal row) stream through shared memory by TMA, and the per-block
//    frequency sum is evaluated by Horner's rule in the step phasor
//    z = exp(+j 2 pi df tau), then rotated by the block seed. Split over
//    antennas with FP64 partial reduction.
// The phase of every term is exact to ~1e-6 rad: r is formed as a
// double-single from the FP32 coordinates, r * 2 f / c is reduced to its
// fractional cycle in double-single before the seed's sincos.
#include <math.h>
#include <stdio.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace geraf {

namespace {

constexpr float kInv16Pi2 = 0.0063325739776461107f;   // 1 / (16 pi^2)
constexpr float kSqrt2 = 1.41421356237309505f;

// ------------------------------------------------------------------ records
// Point record of the phasor kernels (48 bytes); the position is split as
// x = xh + xl (split_coord: xh on the 2^-10 m grid, xl the exact remainder;
// for the Chebyshev kernels in carrier cycles, split_cyc):
//  render / render backward: a = (xh, yh, zh, w), b = (sqrt2*nx, sqrt2*ny, sqrt2*nz, t_eff),
//                            c = (xl, yl, zl, e); e = 1 directional, -1 isotropic
//  filter backward:          a = (xh, yh, zh, c_re), b = (c_im, 0, 0, 0), c = (xl, yl, zl, 0)
struct __align__(16) PtRec {
    float4 a, b, c;
};

// Pair layout of the to-bins Chebyshev records: records 2p and 2p + 1 share
// 96 bytes, field f (a.x .. c.w, in that order) of record 2p + s at float
// 24 p + 2 f + s, so that one 16-byte load gives two fields of both points as
// two packed (f32x2) operands. The render records hold -e in c.w there.
__device__ __forceinline__ void store_rec(PtRec* __restrict__ out, int64_t r, const PtRec& v, bool pair) {
    if (!pair) {
        out[r] = v;
        return;
    }
    float* base = reinterpret_cast<float*>(out) + (r >> 1) * 24 + (r & 1);
    const float f[12] = {v.a.x, v.a.y, v.a.z, v.a.w, v.b.x, v.b.y, v.b.z, v.b.w, v.c.x, v.c.y, v.c.z, v.c.w};
#pragma unroll
    for (int q = 0; q < 12; ++q) base[2 * q] = f[q];
}
// field f of record r in the pair layout
__device__ __forceinline__ float pair_field(const PtRec* __restrict__ pts, int64_t r, int f) {
    return reinterpret_cast<const float*>(pts)[(r >> 1) * 24 + 2 * f + (r & 1)];
}

// 1/|G| of a directional point (0 for an isotropic one), shared by the pack
// kernel and the render adjoint's finalize so both see the same value
__device__ __forceinline__ float inv_grad_norm(float gx, float gy, float gz, int directional) {
    const float g2 = __fmaf_rn(gz, gz, __fmaf_rn(gy, gy, __fmul_rn(gx, gx)));
    return (directional && g2 > 0.0f) ? 1.0f / sqrtf(g2) : 0.0f;
}

__device__ __forceinline__ void split3(float x, float y, float z, float4& hi, float4& lo) {
    split_coord(x, hi.x, lo.x);
    split_coord(y, hi.y, lo.y);
    split_coord(z, hi.z, lo.z);
}

// the same in carrier cycles (split_cyc), for the Chebyshev kernels
__device__ __forceinline__ void split3c(float x, float y, float z, double k0, float4& hi, float4& lo) {
    split_cyc(x, k0, hi.x, lo.x);
    split_cyc(y, k0, hi.y, lo.y);
    split_cyc(z, k0, hi.z, lo.z);
}

// split in cycles when the call runs the Chebyshev kernels (cyc_if not NULL
// and *cyc_if, the plan's run_cheb), else in metres for the recurrence kernels
__device__ __forceinline__ void split3p(float x, float y, float z, const int* cyc_if, double k0, float4& hi,
                                        float4& lo) {
    if (cyc_if && *cyc_if)
        split3c(x, y, z, k0, hi, lo);
    else
        split3(x, y, z, hi, lo);
}

// --------------------------------------------------------------- pack kernels
// record j holds point perm[j] (perm NULL: point j); with pair set, the
// records of a Chebyshev call (*cyc_if) take the pair layout (n_pad even)
__global__ void pack_render_points(const float* __restrict__ xyz, const float* __restrict__ grad,
                                   const float* __restrict__ w, const float* __restrict__ t_eff,
                                   int64_t n, int64_t n_pad, int directional, PtRec* __restrict__ out,
                                   const int* __restrict__ perm = nullptr, const int* cyc_if = nullptr,
                                   double k0 = 0.0, int pair = 0) {
    const int64_t r_ = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r_ >= n_pad) return;
    const bool pl = pair && cyc_if && *cyc_if;
    const int64_t j = r_ < n && perm ? perm[r_] : r_;
    PtRec r;
    if (r_ < n) {
        const float gx = grad[j], gy = grad[n + j], gz = grad[2 * n + j];
        const float ig = inv_grad_norm(gx, gy, gz, directional);
        const bool dir = ig > 0.0f;
        const float k = kSqrt2 * ig;
        split3p(xyz[j], xyz[n + j], xyz[2 * n + j], cyc_if, k0, r.a, r.c);
        r.a.w = w[j];
        r.b = make_float4(gx * k, gy * k, gz * k, t_eff[j]);
        r.c.w = dir ? 1.0f : -1.0f;
    } else {
        // padding: the last point's position with zero weight (inside the
        // range bound of the call and of the last split)
        split3p(xyz[n - 1], xyz[2 * n - 1], xyz[3 * n - 1], cyc_if, k0, r.a, r.c);
        r.a.w = 0.0f;
        r.b = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        r.c.w = -1.0f;
    }
    if (pl) r.c.w = -r.c.w;
    store_rec(out, r_, r, pl);
}

__global__ void pack_filter_bwd_points(const float* __restrict__ vox, const float2* __restrict__ M,
                                       const float* __restrict__ dP, int64_t n, int64_t n_pad,
                                       PtRec* __restrict__ out, const int* __restrict__ perm = nullptr,
                                       const int* cyc_if = nullptr, double k0 = 0.0, int pair = 0) {
    const int64_t r_ = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r_ >= n_pad) return;
    const bool pl = pair && cyc_if && *cyc_if;
    const int64_t j = r_ < n && perm ? perm[r_] : r_;
    PtRec r;
    if (r_ < n) {
        float2 m = M[j];
        double mag = sqrt((double)m.x * m.x + (double)m.y * m.y);
        float cr = 0.0f, ci = 0.0f;
        if (mag > 0.0) {
            cr = (float)(dP[j] * (double)m.x / mag);
            ci = (float)(dP[j] * (double)m.y / mag);
        }
        split3p(vox[j], vox[n + j], vox[2 * n + j], cyc_if, k0, r.a, r.c);
        r.a.w = cr;
        r.b = make_float4(ci, 0.0f, 0.0f, 0.0f);
    } else {
        split3p(vox[n - 1], vox[2 * n - 1], vox[3 * n - 1], cyc_if, k0, r.a, r.c);
        r.a.w = 0.0f;
        r.b = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    r.c.w = 0.0f;
    store_rec(out, r_, r, pl);
}

// antenna records (x, y, z, c_ant), padded with copies of antenna 0
__global__ void pack_antennas(const float* __restrict__ ant, const float* __restrict__ c_ant, int n_ant,
                              int n_pad, float4* __restrict__ out) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_pad) return;
    int k = i < n_ant ? i : 0;
    out[i] = make_float4(ant[k], ant[n_ant + k], ant[2 * n_ant + k], c_ant ? c_ant[k] : 0.0f);
}

// ------------------------------------------------- spatial order of antennas
// The Chebyshev kernels expand each part of a call (points x a block of
// CH_THREADS consecutive antenna records) over the part's own range interval,
// whose width sets the order. Consecutive antennas in the caller's order need
// not be close (a row-major array puts a 128-antenna block on one 25 cm line),
// so the Chebyshev calls pack the antennas in Morton (Z-curve) order of their
// positions, quantised to 10 bits per axis over the array's bounding box (one
// scale for all three axes): on a regular planar grid every block of 128
// records is then a 16 x 8 (or 8 x 16) patch. perm[r] = the antenna held by
// record r; records past n_ant hold antenna 0 and are never written back.
// Keys (code << 32 | index) are unique, so the order is deterministic. One CTA,
// bitonic sort in shared memory up to AO_SMEM_MAX antennas, above that in a
// global scratch buffer (every pass ends with a block barrier).
constexpr int AO_THREADS = 1024;
constexpr int AO_SMEM_MAX = 16384;

__device__ __forceinline__ uint64_t spread3_10(uint32_t v) {
    uint64_t x = v & 0x3FFu;
    x = (x | (x << 16)) & 0x30000FFull;
    x = (x | (x << 8)) & 0x300F00Full;
    x = (x | (x << 4)) & 0x30C30C3ull;
    x = (x | (x << 2)) & 0x9249249ull;
    return x;
}

__global__ void __launch_bounds__(AO_THREADS) antenna_order_kernel(const float* __restrict__ ant, int n_ant,
                                                                   int n_pow2, unsigned long long* __restrict__ gbuf,
                                                                   int* __restrict__ perm, int n_perm) {
    extern __shared__ unsigned long long sbuf[];
    __shared__ float red[6][AO_THREADS / 32];
    unsigned long long* buf = n_pow2 <= AO_SMEM_MAX ? sbuf : gbuf;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int i = t; i < n_ant; i += AO_THREADS)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float v = ant[d * n_ant + i];
            mn[d] = fminf(mn[d], v);
            mx[d] = fmaxf(mx[d], v);
        }
#pragma unroll
    for (int d = 0; d < 3; ++d)
        for (int o = 16; o > 0; o >>= 1) {
            mn[d] = fminf(mn[d], __shfl_xor_sync(0xffffffffu, mn[d], o));
            mx[d] = fmaxf(mx[d], __shfl_xor_sync(0xffffffffu, mx[d], o));
        }
    if (lane == 0)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            red[d][warp] = mn[d];
            red[3 + d][warp] = mx[d];
        }
    __syncthreads();
    float lo[3], span = 0.0f;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        float a = INFINITY, b = -INFINITY;
        for (int w = 0; w < AO_THREADS / 32; ++w) {
            a = fminf(a, red[d][w]);
            b = fmaxf(b, red[3 + d][w]);
        }
        lo[d] = a;
        span = fmaxf(span, b - a);
    }
    const float scale = span > 0.0f ? 1023.0f / span : 0.0f;
    for (int i = t; i < n_pow2; i += AO_THREADS) {
        unsigned long long key = ~0ull;
        if (i < n_ant) {
            uint64_t code = 0;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const float q = fminf(fmaxf((ant[d * n_ant + i] - lo[d]) * scale, 0.0f), 1023.0f);
                code |= spread3_10((uint32_t)q) << d;
            }
            key = (code << 32) | (unsigned long long)(uint32_t)i;
        }
        buf[i] = key;
    }
    __syncthreads();
    for (int k = 2; k <= n_pow2; k <<= 1)
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int i = t; i < n_pow2; i += AO_THREADS) {
                const int l = i ^ j;
                if (l > i) {
                    const unsigned long long a = buf[i], b = buf[l];
                    if ((a > b) == ((i & k) == 0)) {
                        buf[i] = b;
                        buf[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (int r = t; r < n_perm; r += AO_THREADS) perm[r] = r < n_ant ? (int)(uint32_t)(buf[r] & 0xffffffffull) : 0;
}

size_t antenna_order_smem(int n_pow2) { return n_pow2 <= AO_SMEM_MAX ? (size_t)n_pow2 * 8 : 0; }
int pow2_at_least(int n) {
    int p = 1;
    while (p < n) p <<= 1;
    return p;
}

// antenna records (x, y, z, c_ant) in the spatial order perm (records past
// n_ant hold antenna 0)
__global__ void pack_antennas_perm(const float* __restrict__ ant, const float* __restrict__ c_ant, int n_ant,
                                   const int* __restrict__ perm, int n_pad, float4* __restrict__ out) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_pad) return;
    const int k = perm[r];
    out[r] = make_float4(ant[k], ant[n_ant + k], ant[2 * n_ant + k], c_ant ? c_ant[k] : 0.0f);
}

// antenna tile rows for the to-points kernels: 16-byte head (x, y, z, c)
// followed by one float4 (s_re, s_re, s_im, s_im) per bin, zero-padded to
// 32*G bins, so that one 16-byte load gives the packed pairs (s_re, s_re)
// and (s_im, s_im) of the two-lane Horner sums.
__global__ void pack_antenna_rows(const float* __restrict__ ant, const float* __restrict__ c_ant,
                                  const float2* __restrict__ sig, int n_ant, int n_ant_pad, int n_f,
                                  int n_f_pad, float4* __restrict__ out, const int* run_if = nullptr) {
    if (run_if && *run_if == 0) return;
    int i = blockIdx.x;
    if (i >= n_ant_pad) return;
    float4* row = out + (size_t)i * (1 + n_f_pad);
    if (threadIdx.x == 0) {
        int k = i < n_ant ? i : 0;
        row[0] = make_float4(ant[k], ant[n_ant + k], ant[2 * n_ant + k], c_ant ? c_ant[k] : 0.0f);
    }
    for (int n = threadIdx.x; n < n_f_pad; n += blockDim.x) {
        float2 v = make_float2(0.0f, 0.0f);
        if (i < n_ant && n < n_f) v = sig[(size_t)i * n_f + n];
        row[1 + n] = make_float4(v.x, v.x, v.y, v.y);
    }
}

// ------------------------------------------------------------ to-bins kernel
constexpr int TB_THREADS = 128;
constexpr int TB_FLUSH_TILES = 4;

struct ToBinsArgs {
    const PtRec* pts;        // n_tiles * tp records
    const float4* ant;       // n_ant_pad records
    float2* partial;         // [splits][n_ant_pad][32 G]
    int* err;
    int tp;                  // points per tile (8, 16 or 32; even)
    int n_tiles;             // total point tiles
    int tiles_per_split;
    int n_ant_pad;
    int a_t;                 // antennas per CTA
    BandK bk;
    const int* run_if;       // when set, the kernel runs only if *run_if != 0
};

template <bool kComplexAmp>
__global__ void __launch_bounds__(TB_THREADS, 2) to_bins_kernel(const ToBinsArgs args) {
    if (args.run_if && *args.run_if == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    const int G = args.bk.g;
    const int A_T = args.a_t;
    const int TP = args.tp;
    const int t = threadIdx.x;

    // shared layout
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);                       // 2 barriers
    int* abort_flag = reinterpret_cast<int*>(smem + 16);
    PtRec* tiles = reinterpret_cast<PtRec*>(smem + 32);                      // [2][TP]
    float4* ant_s = reinterpret_cast<float4*>(smem + 32 + 2 * TP * sizeof(PtRec));
    float* prep = reinterpret_cast<float*>(ant_s + A_T);                     // [6][TP][A_T]
    float2* outer = reinterpret_cast<float2*>(prep + 6 * TP * A_T);          // [2][32][TB_THREADS]

    const int ant0 = blockIdx.x * A_T;
    const int split = blockIdx.y;
    const int tile0 = split * args.tiles_per_split;
    const int tile1 = min(tile0 + args.tiles_per_split, args.n_tiles);
    const int n_my = tile1 - tile0;

    const int a_slot = t / G;
    const int blk = t - a_slot * G;
    const bool active = a_slot < A_T;

    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    for (int i = t; i < A_T; i += TB_THREADS) ant_s[i] = args.ant[ant0 + i];
    for (int i = t; i < 2 * 32 * TB_THREADS; i += TB_THREADS) outer[i] = make_float2(0.0f, 0.0f);
    __syncthreads();

    const uint32_t tile_bytes = (uint32_t)(TP * sizeof(PtRec));
    if (t == 0) {
        for (int s = 0; s < 2 && s < n_my; ++s) {
            mbar_arrive_expect_tx(&bar[s], tile_bytes);
            tma_load_1d(tiles + s * TP, args.pts + (size_t)(tile0 + s) * TP, tile_bytes, &bar[s]);
        }
    }

    const float kh = args.bk.k[2 * blk], kl = args.bk.k[2 * blk + 1];
    const float kd = args.bk.kd;
    // accumulators of bins 32 blk + m: lanes = even / odd points of the tile
    f2 accr[32], acci[32];
#pragma unroll
    for (int m = 0; m < 32; ++m) accr[m] = acci[m] = 0ull;

    for (int it = 0; it < n_my; ++it) {
        const int buf = it & 1;
        bool ok = mbar_wait(&bar[buf], (it >> 1) & 1);
        if (!ok) atomicOr(abort_flag, 1);
        __syncthreads();
        if (*abort_flag) {
            if (t == 0) {
                atomicOr(args.err, 1);
                mbar_drain2(bar, it, n_my);
            }
            return;
        }
        const PtRec* tile = tiles + buf * TP;
        // ---- per-pair preparation shared by the G bin blocks of an antenna
        for (int q = t; q < TP * A_T; q += TB_THREADS) {
            const int p = q / A_T, a = q - p * A_T;
            const PtRec P = tile[p];
            const float4 A4 = ant_s[a];
            Range R = pair_range(P.a.x + P.c.x, P.a.y + P.c.y, P.a.z + P.c.z, A4.x, A4.y, A4.z);
            float amp = 0.0f;
            if (!kComplexAmp) {
                float inv_r2 = R.rs * R.rs;
                float nd = P.b.x * R.dx + P.b.y * R.dy + P.b.z * R.dz;
                float D = fmaxf(nd * nd * inv_r2 - P.c.w, 0.0f);
                float tt = __saturatef(P.b.w - A4.w);
                amp = P.a.w * tt * tt * (inv_r2 * kInv16Pi2) * D;
            } else {
                amp = P.a.w;         // c_re (c_im goes to prep row 5)
            }
            float dl = R.rh * kd;
            dl = dl - rintf(dl);
            float sn, cs;
            sincospif(2.0f * dl, &sn, &cs);
            prep[(0 * TP + p) * A_T + a] = R.rh;
            prep[(1 * TP + p) * A_T + a] = R.rl;
            prep[(2 * TP + p) * A_T + a] = amp;
            prep[(3 * TP + p) * A_T + a] = cs;
            prep[(4 * TP + p) * A_T + a] = -sn;     // step exp(-j 2 pi delta)
            if (kComplexAmp) prep[(5 * TP + p) * A_T + a] = P.b.x;
        }
        __syncthreads();
        // ---- 32-bin recurrence per (point pair, my antenna, my block), packed f32x2
        if (active) {
            for (int p = 0; p < TP; p += 2) {
                float qr[2], qi[2], wr[2], wi[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float rh = prep[(0 * TP + p + h) * A_T + a_slot];
                    const float rl = prep[(1 * TP + p + h) * A_T + a_slot];
                    wr[h] = prep[(3 * TP + p + h) * A_T + a_slot];
                    wi[h] = prep[(4 * TP + p + h) * A_T + a_slot];
                    const float fr = phase_frac(rh, rl, kh, kl);
                    float sn, cs;
                    __sincosf(6.28318530717958648f * fr, &sn, &cs);
                    const float amp = prep[(2 * TP + p + h) * A_T + a_slot];
                    if (!kComplexAmp) {
                        qr[h] = amp * cs;
                        qi[h] = -amp * sn;
                    } else {
                        const float ci = prep[(5 * TP + p + h) * A_T + a_slot];
                        // (c_re + j c_im)(cs - j sn)
                        qr[h] = amp * cs + ci * sn;
                        qi[h] = ci * cs - amp * sn;
                    }
                }
                f2 Qr = pk2(qr[0], qr[1]), Qi = pk2(qi[0], qi[1]);
                const f2 Wr = pk2(wr[0], wr[1]), Wi = pk2(wi[0], wi[1]), NWi = pk2(-wi[0], -wi[1]);
#pragma unroll
                for (int m = 0; m < 32; ++m) {
                    accr[m] = add2(accr[m], Qr);
                    acci[m] = add2(acci[m], Qi);
                    const f2 t1 = mul2(Qi, NWi);
                    const f2 t2 = mul2(Qi, Wr);
                    const f2 nr = fma2(Qr, Wr, t1);
                    Qi = fma2(Qr, Wi, t2);
                    Qr = nr;
                }
            }
        }
        // ---- Kahan flush of the inner sums (both lanes)
        if (active && (((it + 1) % TB_FLUSH_TILES) == 0 || it + 1 == n_my)) {
#pragma unroll
            for (int m = 0; m < 32; ++m) {
                float r0, r1, i0, i1;
                upk2(accr[m], r0, r1);
                upk2(acci[m], i0, i1);
                float2 hi = outer[m * TB_THREADS + t];
                float2 lo = outer[(32 + m) * TB_THREADS + t];
                float yx = __fsub_rn(__fadd_rn(r0, r1), lo.x), yy = __fsub_rn(__fadd_rn(i0, i1), lo.y);
                float sx = __fadd_rn(hi.x, yx), sy = __fadd_rn(hi.y, yy);
                lo.x = __fsub_rn(__fsub_rn(sx, hi.x), yx);
                lo.y = __fsub_rn(__fsub_rn(sy, hi.y), yy);
                outer[m * TB_THREADS + t] = make_float2(sx, sy);
                outer[(32 + m) * TB_THREADS + t] = lo;
                accr[m] = acci[m] = 0ull;
            }
        }
        __syncthreads();   // tile and prep buffers are free again
        if (t == 0 && it + 2 < n_my) {
            mbar_arrive_expect_tx(&bar[buf], tile_bytes);
            tma_load_1d(tiles + buf * TP, args.pts + (size_t)(tile0 + it + 2) * TP, tile_bytes, &bar[buf]);
        }
    }
    if (active) {
        const int n_f_pad = 32 * G;
        float2* dst = args.partial + ((size_t)split * args.n_ant_pad + ant0 + a_slot) * n_f_pad + 32 * blk;
#pragma unroll
        for (int m = 0; m < 32; ++m) {
            float2 hi = outer[m * TB_THREADS + t];
            float2 lo = outer[(32 + m) * TB_THREADS + t];
            dst[m] = make_float2(__fsub_rn(hi.x, lo.x), __fsub_rn(hi.y, lo.y));
        }
    }
}

// partial [splits][n_ant_pad][n_f_pad] -> out [n_ant][n_f], FP64 sum in split order
__global__ void reduce_bins(const float2* __restrict__ partial, int splits, int n_ant, int n_ant_pad, int n_f,
                            int n_f_pad, float2* __restrict__ out, const int* run_if = nullptr) {
    if (run_if && *run_if == 0) return;
    int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n_ant * n_f) return;
    int i = (int)(idx / n_f), n = (int)(idx - (int64_t)i * n_f);
    double sr = 0.0, si = 0.0;
    for (int s = 0; s < splits; ++s) {
        float2 v = partial[((size_t)s * n_ant_pad + i) * n_f_pad + n];
        sr += v.x;
        si += v.y;
    }
    out[idx] = make_float2((float)sr, (float)si);
}

// ----------------------------------------------------------- to-points kernel
constexpr int TPK_THREADS = 128;
constexpr int TPK_V = 2;          // points per thread = the two lanes of the packed Horner sums

enum { MODE_FILTER = 0, MODE_RENDER_BWD = 1 };

struct ToPointsArgs {
    const PtRec* pts;          // padded point records (render backward)
    const float* vox;          // [3][n] voxel positions (filter)
    int64_t n;                 // points / voxels
    const float4* rows;        // antenna rows: head (x, y, z, c) + per bin (s_re, s_re, s_im, s_im)
    int row_f4;                // float4 per antenna row = 1 + n_f_pad
    int at;                    // antennas per tile
    int n_ant_tiles;
    int tiles_per_split;
    float* partial;            // filter: float2 [splits][n]; render bwd: float [splits][6][n]
    int* err;
    BandK bk;
    const int* run_if;         // when set, the kernel runs only if *run_if != 0
};

template <int MODE>
__global__ void __launch_bounds__(TPK_THREADS) to_points_kernel(const ToPointsArgs args) {
    if (args.run_if && *args.run_if == 0) return;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int* abort_flag = reinterpret_cast<int*>(smem + 16);
    float4* rows = reinterpret_cast<float4*>(smem + 32);   // [2][at][row_f4]
    const int G = args.bk.g;
    const int row_f4 = args.row_f4;
    const int AT = args.at;
    const int t = threadIdx.x;
    const int split = blockIdx.y;
    const int tile0 = split * args.tiles_per_split;
    const int tile1 = min(tile0 + args.tiles_per_split, args.n_ant_tiles);
    const int n_my = tile1 - tile0;
    const uint32_t tile_bytes = (uint32_t)(AT * row_f4 * sizeof(float4));

    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (t == 0) {
        for (int s = 0; s < 2 && s < n_my; ++s) {
            mbar_arrive_expect_tx(&bar[s], tile_bytes);
            tma_load_1d(rows + s * AT * row_f4, args.rows + (size_t)(tile0 + s) * AT * row_f4, tile_bytes, &bar[s]);
        }
    }

    // my points
    const int64_t jbase = (blockIdx.x * (int64_t)TPK_THREADS + t) * TPK_V;
    float px[TPK_V], py[TPK_V], pz[TPK_V];
    float pw[TPK_V], pnx[TPK_V], pny[TPK_V], pnz[TPK_V], pte[TPK_V], pe[TPK_V];
#pragma unroll
    for (int v = 0; v < TPK_V; ++v) {
        const int64_t j = min(jbase + v, args.n - 1);
        if (MODE == MODE_FILTER) {
            px[v] = args.vox[j];
            py[v] = args.vox[args.n + j];
            pz[v] = args.vox[2 * args.n + j];
            pw[v] = pnx[v] = pny[v] = pnz[v] = pte[v] = pe[v] = 0.0f;
        } else {
            const PtRec P = args.pts[j];
            px[v] = P.a.x + P.c.x; py[v] = P.a.y + P.c.y; pz[v] = P.a.z + P.c.z; pw[v] = P.a.w;
            pnx[v] = P.b.x; pny[v] = P.b.y; pnz[v] = P.b.z; pte[v] = P.b.w;
            pe[v] = P.c.w;
        }
    }
    // outer (Kahan) accumulators; filter: M (re, im); render bwd: d_w, d_teff, Ud(3), Un
    constexpr int NACC = (MODE == MODE_FILTER) ? 2 : 6;
    float hi[TPK_V][NACC], lo[TPK_V][NACC];
#pragma unroll
    for (int v = 0; v < TPK_V; ++v)
#pragma unroll
        for (int k = 0; k < NACC; ++k) hi[v][k] = lo[v][k] = 0.0f;

    const float kd = args.bk.kd;
    for (int it = 0; it < n_my; ++it) {
        const int buf = it & 1;
        bool ok = mbar_wait(&bar[buf], (it >> 1) & 1);
        if (!ok) atomicOr(abort_flag, 1);
        __syncthreads();
        if (*abort_flag) {
            if (t == 0) {
                atomicOr(args.err, 1);
                mbar_drain2(bar, it, n_my);
            }
            return;
        }
        const float4* tile = rows + buf * AT * row_f4;
        float in[TPK_V][NACC];
#pragma unroll
        for (int v = 0; v < TPK_V; ++v)
#pragma unroll
            for (int k = 0; k < NACC; ++k) in[v][k] = 0.0f;

        for (int a = 0; a < AT; ++a) {
            const float4 head = tile[a * row_f4];
            const ulonglong2* sig = reinterpret_cast<const ulonglong2*>(tile + a * row_f4 + 1);
            Range R[TPK_V];
            float zr[TPK_V], zi[TPK_V], hr[TPK_V], him[TPK_V];
#pragma unroll
            for (int v = 0; v < TPK_V; ++v) {
                R[v] = pair_range(px[v], py[v], pz[v], head.x, head.y, head.z);
                float dl = R[v].rh * kd;
                dl = dl - rintf(dl);
                float sn, cs;
                sincospif(2.0f * dl, &sn, &cs);
                zr[v] = cs;
                zi[v] = sn;      // z = exp(+j 2 pi delta)
                hr[v] = 0.0f;
                him[v] = 0.0f;
            }
            const f2 Zr = pk2(zr[0], zr[1]), Zi = pk2(zi[0], zi[1]), NZi = pk2(-zi[0], -zi[1]);
            for (int b = 0; b < G; ++b) {
                const float kh = args.bk.k[2 * b], kl = args.bk.k[2 * b + 1];
                const ulonglong2* sb = sig + 32 * b;
                // Horner: sum_m s_m z^m, both points at once (lanes), s broadcast to both lanes
                const ulonglong2 top = sb[31];
                f2 Ar = top.x, Ai = top.y;
#pragma unroll
                for (int m = 30; m >= 0; --m) {
                    const ulonglong2 sv = sb[m];
                    const f2 t1 = fma2(Ai, NZi, sv.x);
                    const f2 t2 = fma2(Ai, Zr, sv.y);
                    const f2 nr = fma2(Ar, Zr, t1);
                    Ai = fma2(Ar, Zi, t2);
                    Ar = nr;
                }
                float ar[TPK_V], ai[TPK_V];
                upk2(Ar, ar[0], ar[1]);
                upk2(Ai, ai[0], ai[1]);
#pragma unroll
                for (int v = 0; v < TPK_V; ++v) {
                    const float fr = phase_frac(R[v].rh, R[v].rl, kh, kl);
                    float sn, cs;
                    __sincosf(6.28318530717958648f * fr, &sn, &cs);
                    // seed exp(+j 2 pi psi_b) times the block's Horner sum
                    hr[v] = fmaf(cs, ar[v], fmaf(-sn, ai[v], hr[v]));
                    him[v] = fmaf(cs, ai[v], fmaf(sn, ar[v], him[v]));
                }
            }
#pragma unroll
            for (int v = 0; v < TPK_V; ++v) {
                if (MODE == MODE_FILTER) {
                    in[v][0] += hr[v];
                    in[v][1] += him[v];
                } else {
                    // q = Re(sum_n g e^{+j phi}); gradients of A = w T'^2 gamma D
                    const float q = hr[v];
                    const float inv_r2 = R[v].rs * R[v].rs;
                    const float gam = inv_r2 * kInv16Pi2;
                    const float nd = pnx[v] * R[v].dx + pny[v] * R[v].dy + pnz[v] * R[v].dz;
                    const float c2x2 = nd * nd * inv_r2;          // 2 c^2 (0 when isotropic)
                    const float Dm = c2x2 - pe[v];
                    const float D = fmaxf(Dm, 0.0f);
                    const float vv = pte[v] - head.w;
                    const float tt = __saturatef(vv);
                    const float gq = gam * q;
                    in[v][0] += tt * tt * D * gq;
                    if (vv >= 0.0f && vv <= 1.0f) in[v][1] += pw[v] * 2.0f * tt * D * gq;
                    if (pe[v] > 0.0f && Dm > 0.0f) {
                        // dD/dG = 4 c (w_i - c n)/|G|, c = nd / (sqrt2 r): split into
                        // Ud += k 4 c / r * d  and  Un += k 4 c^2 / sqrt2 (times n' later)
                        const float kq = pw[v] * tt * tt * gq;
                        const float c = nd * R[v].rs * (1.0f / kSqrt2);
                        const float k1 = kq * 4.0f * c * R[v].rs;
                        in[v][2] += k1 * R[v].dx;
                        in[v][3] += k1 * R[v].dy;
                        in[v][4] += k1 * R[v].dz;
                        in[v][5] += kq * 4.0f * c * c * (1.0f / kSqrt2);
                    }
                }
            }
        }
        // Kahan accumulate the tile's inner sums
#pragma unroll
        for (int v = 0; v < TPK_V; ++v)
#pragma unroll
            for (int k = 0; k < NACC; ++k) {
                const float y = __fsub_rn(in[v][k], lo[v][k]);
                const float s = __fadd_rn(hi[v][k], y);
                lo[v][k] = __fsub_rn(__fsub_rn(s, hi[v][k]), y);
                hi[v][k] = s;
            }
        __syncthreads();
        if (t == 0 && it + 2 < n_my) {
            mbar_arrive_expect_tx(&bar[buf], tile_bytes);
            tma_load_1d(rows + buf * AT * row_f4, args.rows + (size_t)(tile0 + it + 2) * AT * row_f4, tile_bytes,
                        &bar[buf]);
        }
    }
#pragma unroll
    for (int v = 0; v < TPK_V; ++v) {
        const int64_t j = jbase + v;
        if (j >= args.n) continue;
        if (MODE == MODE_FILTER) {
            float2* dst = reinterpret_cast<float2*>(args.partial) + (size_t)split * args.n + j;
            *dst = make_float2(__fsub_rn(hi[v][0], lo[v][0]), __fsub_rn(hi[v][1], lo[v][1]));
        } else {
            float* dst = args.partial + (size_t)split * 6 * args.n + j;
#pragma unroll
            for (int k = 0; k < 6; ++k) dst[(size_t)k * args.n] = __fsub_rn(hi[v][k], lo[v][k]);
        }
    }
}

// filter finalize: M = sum of split partials (FP64), P = |M|, loss terms
// record j -> voxel o = perm[j] (perm NULL: o = j)
__global__ void filter_finalize(const float2* __restrict__ partial, int splits, int64_t n,
                                const float* __restrict__ target, const float* __restrict__ mask,
                                float* __restrict__ P, float2* __restrict__ M, float* __restrict__ dP,
                                double* __restrict__ loss_blocks, const int* __restrict__ perm) {
    __shared__ double red[256];
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double l = 0.0;
    if (j < n) {
        const int64_t o = perm ? perm[j] : j;
        double mr = 0.0, mi = 0.0;
        for (int s = 0; s < splits; ++s) {
            float2 v = partial[(size_t)s * n + j];
            mr += v.x;
            mi += v.y;
        }
        double p = sqrt(mr * mr + mi * mi);
        M[o] = make_float2((float)mr, (float)mi);
        P[o] = (float)p;
        if (target) {
            double m = mask ? (double)mask[o] : 1.0;
            double r = p - (double)target[o];
            l = m * r * r;
            if (dP) dP[o] = (float)(2.0 * m * r);
        }
    }
    if (loss_blocks) {
        red[threadIdx.x] = l;
        __syncthreads();
        for (int s = blockDim.x / 2; s > 0; s >>= 1) {
            if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
            __syncthreads();
        }
        if (threadIdx.x == 0) loss_blocks[blockIdx.x] = red[0];
    }
}

__global__ void sum_doubles(const double* __restrict__ x, int n, double* __restrict__ out) {
    __shared__ double red[256];
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = red[0];
}

// record j -> point o = perm[j] (perm NULL: o = j)
__global__ void render_bwd_finalize(const float* __restrict__ partial, int splits, int64_t n,
                                    const PtRec* __restrict__ pts, const float* __restrict__ grad,
                                    int directional, float* __restrict__ d_w,
                                    float* __restrict__ d_teff, float* __restrict__ d_grad,
                                    const int* __restrict__ perm) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t o = perm ? perm[j] : j;
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int s = 0; s < splits; ++s)
        for (int k = 0; k < 6; ++k) acc[k] += partial[((size_t)s * 6 + k) * n + j];
    d_w[o] = (float)acc[0];
    d_teff[o] = (float)acc[1];
    const PtRec P = pts[j];
    const double ig = inv_grad_norm(grad[o], grad[n + o], grad[2 * n + o], directional);   // 0 when isotropic
    d_grad[o] = (float)((acc[2] - acc[5] * P.b.x) * ig);
    d_grad[n + o] = (float)((acc[3] - acc[5] * P.b.y) * ig);
    d_grad[2 * n + o] = (float)((acc[4] - acc[5] * P.b.z) * ig);
}

// --------------------------------------------------------------- launch glue

int choose_splits(int64_t base_ctas, int resident_per_sm, int64_t max_splits) {
    const int64_t slots = (int64_t)device_sm_count() * resident_per_sm;
    int64_t waves = (base_ctas + slots - 1) / slots;
    if (waves < 4) waves = 4;
    int64_t s = (waves * slots + base_ctas - 1) / base_ctas;
    if (s > max_splits) s = max_splits;
    if (s < 1) s = 1;
    return (int)s;
}

struct ToBinsPlan {
    int G, A_T, TP, n_ant_pad, ant_ctas, n_tiles, splits, tiles_per_split;
    size_t smem;
};

ToBinsPlan plan_to_bins(int64_t n_pts, int n_ant, int G) {
    ToBinsPlan p;
    p.G = G;
    p.A_T = TB_THREADS / G;
    if (p.A_T < 1) p.A_T = 1;
    p.TP = (p.A_T >= 128) ? 8 : (p.A_T >= 64 ? 16 : 32);   // prep rows <= 32 KB, two CTAs per SM
    p.n_ant_pad = (int)((n_ant + p.A_T - 1) / p.A_T) * p.A_T;
    p.ant_ctas = p.n_ant_pad / p.A_T;
    p.n_tiles = (int)((n_pts + p.TP - 1) / p.TP);
    if (p.n_tiles < 1) p.n_tiles = 1;
    p.splits = choose_splits(p.ant_ctas, 2, p.n_tiles);
    p.tiles_per_split = (p.n_tiles + p.splits - 1) / p.splits;
    p.splits = (p.n_tiles + p.tiles_per_split - 1) / p.tiles_per_split;
    p.smem = 32 + 2 * p.TP * sizeof(PtRec) + p.A_T * sizeof(float4) + 6 * p.TP * p.A_T * sizeof(float) +
             2 * 32 * TB_THREADS * sizeof(float2);
    return p;
}

struct ToPointsPlan {
    int G, n_f_pad, row_f4, at, n_ant_pad, n_ant_tiles, pt_ctas, splits, tiles_per_split;
    size_t smem;
};

ToPointsPlan plan_to_points(int64_t n, int n_ant, int G) {
    ToPointsPlan p;
    p.G = G;
    p.n_f_pad = 32 * G;
    p.row_f4 = 1 + p.n_f_pad;
    p.at = G <= 8 ? 8 : (G <= 16 ? 4 : 2);     // two tiles <= ~132 KB of shared memory
    p.n_ant_pad = (n_ant + p.at - 1) / p.at * p.at;
    p.n_ant_tiles = p.n_ant_pad / p.at;
    p.pt_ctas = (int)((n + TPK_THREADS * TPK_V - 1) / (TPK_THREADS * TPK_V));
    p.splits = choose_splits(p.pt_ctas, 8, p.n_ant_tiles);
    p.tiles_per_split = (p.n_ant_tiles + p.splits - 1) / p.splits;
    p.splits = (p.n_ant_tiles + p.tiles_per_split - 1) / p.tiles_per_split;
    p.smem = 32 + 2 * (size_t)p.at * p.row_f4 * sizeof(float4);
    return p;
}

// Antenna tiles of the Chebyshev to-points kernels: CH_PT_AT rows of 1 KB
// (the per-bin recurrence kernels' rows hold every bin and take p.at), with
// the same splits of the antenna tiles as the recurrence plan, so both
// paths leave p.splits partials per point (a split with no tiles writes
// zeros).
struct ChebPointsTiles {
    int at, n_ant_pad, n_ant_tiles, tiles_per_split;
};
constexpr int CH_PT_AT = 16;
ChebPointsTiles cheb_points_tiles(const ToPointsPlan& p, int n_ant) {
    ChebPointsTiles q;
    q.at = CH_PT_AT;
    q.n_ant_pad = std::max(p.n_ant_pad, (n_ant + CH_PT_AT - 1) / CH_PT_AT * CH_PT_AT);
    q.n_ant_tiles = q.n_ant_pad / CH_PT_AT;
    q.tiles_per_split = (q.n_ant_tiles + p.splits - 1) / p.splits;
    return q;
}

// ==================================================== Chebyshev phasor sums
// Per antenna i, the frequency dependence of a term is exp(-j 2 pi f_n 2 r / c)
// with f_n = f_c + m df, f_c the band's centre and m = n - (n_f - 1) / 2. The
// f_c part (K0 = 2 f_c / c, carrier cycles per metre; ranges R = K0 r in
// cycles) is folded into the point's complex amplitude (one double-single
// phase and one sincos per pair); with R = r_c(i) + dr x, |x| <= 1 over a
// range interval centred on each antenna's own ranges, the Jacobi-Anger
// expansion
//   exp(-j a_m x) = sum_k eps_k (-j)^k J_k(a_m) T_k(x),  a_m = 2 pi m Kc dr,
// Kc = df / f_c (bin phase step in cycles per cycle of range), truncated where
// the Bessel tail falls below CH_TAIL, turns the bin sums into K Chebyshev
// moments per antenna (K ~ |a_m|max + 15, about 25 for a 4 GHz sweep over a
// 15 cm range spread, independent of the number of bins):
//   to bins:   s(i, n) = exp(-j 2 pi m Kc r_c(i)) sum_k B_k(m) M_k(i),
//              M_k(i) = sum_j A'_ij T_k(x_ij)
//   to points: sum_n s(i, n) exp(+j ...) = exp(+j 2 pi R) sum_k T_k(x) S_k(i),
//              evaluated per pair with T_k from the three-term recurrence.
// The centred band halves the largest Bessel argument against a band-edge
// carrier, and the per-antenna centre leaves only the part's own extent along
// each antenna's line of sight in the half range dr, not the spread of ranges
// across a block of antennas. Each part of a call (a split of point tiles,
// possibly times a block of antennas, to bins; a group of points, to points)
// has its own half range, order and table B_k(m) = eps_k (-j)^k J_k(a_m),
// computed on the device from the part's bounding box and antennas, so the
// call stays asynchronous; the phase exp(-j 2 pi m Kc r_c(i)) is applied per
// (part, antenna, bin) where the moments meet the bins. If the whole call's
// order K would exceed CH_KMAX the exact recurrence kernels run instead
// (decided on the device).
constexpr int CH_KMAX = 64;
// resident CTAs per SM asked of the compiler for the K <= 32 instances
#ifndef GERAF_CH_BINS_CTAS
#define GERAF_CH_BINS_CTAS 5
#endif
// the render's K <= 24 instance: four (the packed two-point body; six, five and
// four measured 50.5, 49.1 and 48.0 ms on 2^20 points x the 128 x 128 array;
// unrolling two record pairs at four, 49.1)
#ifndef GERAF_CH_BINS_CTAS_24
#define GERAF_CH_BINS_CTAS_24 4
#endif
#ifndef GERAF_CH_FILTER_CTAS
#define GERAF_CH_FILTER_CTAS 8
#endif
#ifndef GERAF_CH_RBWD_CTAS
#define GERAF_CH_RBWD_CTAS 4
#endif
// unroll factors of the per-tile loops (two points of a record tile to bins,
// one antenna row to points); unrolling two antenna rows to points measured
// 64.0 against 63.2 ms on 2^20 points x the 128 x 128 array
#ifndef GERAF_CH_BINS_UNROLL
#define GERAF_CH_BINS_UNROLL 1
#endif
#ifndef GERAF_CH_PTS_UNROLL
#define GERAF_CH_PTS_UNROLL 1
#endif
constexpr int kBinsUnroll = GERAF_CH_BINS_UNROLL;
constexpr int kPtsUnroll = GERAF_CH_PTS_UNROLL;
constexpr int CH_THREADS = 128;
// record tiles of 128 points, the register sums flushed every 256 points
// (tiles of 32, 64 and 128 measured 47.6, 47.2 and 47.1 ms for the render on
// 2^20 points x the 128 x 128 array: fewer CTA barriers per pair)
#ifndef GERAF_CH_TP
#define GERAF_CH_TP 128
#endif
#ifndef GERAF_CH_FLUSH
#define GERAF_CH_FLUSH 2
#endif
constexpr int CH_TP = GERAF_CH_TP;        // points per TMA tile (even: the pair layout)
constexpr int CH_FLUSH = GERAF_CH_FLUSH;  // tiles per inner (register) sum before it joins the outer sum
static_assert(CH_TP % 2 == 0 && CH_TP % 16 == 0, "record tiles hold whole pairs and 16-byte rows");
// Part sizes of the Chebyshev sums. Smaller parts mean narrower range
// intervals and lower orders, at the cost of more split partials, coefficient
// tables and (to points) antenna rows; the byte caps bound those buffers.
#ifndef GERAF_CH_PARTIAL_MIB
#define GERAF_CH_PARTIAL_MIB 6144
#endif
#ifndef GERAF_CH_TABLE_MIB
#define GERAF_CH_TABLE_MIB 12288
#endif
#ifndef GERAF_CH_MAX_SPLITS
#define GERAF_CH_MAX_SPLITS 512
#endif
#ifndef GERAF_CH_SPLIT_CTAS_PER_SM
#define GERAF_CH_SPLIT_CTAS_PER_SM 16
#endif
#ifndef GERAF_CH_SPLIT_MIN_PTS
#define GERAF_CH_SPLIT_MIN_PTS 8192
#endif
// point groups of the to-points sums: up to 512 (one brick each at 2^24
// points: render adjoint 8.2 orders per pair and 796 ms against 9.8 and 821 ms
// with 256 groups of two bricks), at most 16 GiB of antenna rows
#ifndef GERAF_CH_MAX_GROUPS
#define GERAF_CH_MAX_GROUPS 512
#endif
#ifndef GERAF_CH_GROUP_ROWS_MIB
#define GERAF_CH_GROUP_ROWS_MIB 16384
#endif
constexpr size_t CH_PARTIAL_BYTES = (size_t)GERAF_CH_PARTIAL_MIB << 20;   // bound on the split partials of one call
constexpr size_t CH_TABLE_BYTES = (size_t)GERAF_CH_TABLE_MIB << 20;       // bound on the coefficient tables of one call's parts
// Bessel-tail bound of the expansion: the unit phasor is represented to 1e-7,
// below the FP32 rounding of the sums themselves (relative L2 2e-7 .. 5e-7
// against the FP64 oracle on every parity case)
constexpr double CH_TAIL = 1e-7;

struct ChebPlan {
    float inv_dr;     // 1 / the whole set's half range (largest over the antennas), metres
    int K;            // Chebyshev order
    int use_direct;   // 1: the exact recurrence kernels must run instead
    int run_cheb;     // = !use_direct
    float box[6];     // the points' bounding box (min xyz, max xyz)
    int pad;
};

__global__ void bbox_partial_kernel(const float* __restrict__ xyz, int64_t n, float* __restrict__ part) {
    __shared__ float red[6][256];
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x)
        for (int d = 0; d < 3; ++d) {
            const float v = xyz[d * n + j];
            mn[d] = fminf(mn[d], v);
            mx[d] = fmaxf(mx[d], v);
        }
    for (int d = 0; d < 3; ++d) {
        red[d][threadIdx.x] = mn[d];
        red[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k)
            for (int d = 0; d < 3; ++d) {
                red[d][threadIdx.x] = fminf(red[d][threadIdx.x], red[d][threadIdx.x + k]);
                red[3 + d][threadIdx.x] = fmaxf(red[3 + d][threadIdx.x], red[3 + d][threadIdx.x + k]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) part[blockIdx.x * 6 + threadIdx.x] = red[threadIdx.x][0];
}

// J_0 .. J_{kcount-1}(a) by Miller's backward recurrence (normalised by
// J_0 + 2 sum J_2m = 1), FP64
__device__ void bessel_j(double a, int kcount, double* out) {
    if (a < 1e-300) {
        for (int k = 0; k < kcount; ++k) out[k] = k == 0 ? 1.0 : 0.0;
        return;
    }
    int start = kcount + 20 + (int)a;
    start += start & 1;
    const double inv_a2 = 2.0 / a;    // the one division: FP64 divides are long on this part
    double jp1 = 0.0, j = 1e-300, norm = 0.0;
    for (int k = start; k >= 1; --k) {
        const double jm1 = ((double)k * inv_a2) * j - jp1;
        jp1 = j;
        j = jm1;                      // j = J_{k-1}
        if (k - 1 < kcount) out[k - 1] = j;
        if ((k - 1) % 2 == 0 && k - 1 > 0) norm += 2.0 * j;
        if (fabs(j) > 1e250) {        // rescale
            jp1 *= 1e-250;
            j *= 1e-250;
            norm *= 1e-250;
            for (int q = k - 1; q < kcount; ++q) out[q] *= 1e-250;
        }
    }
    norm += j;                        // J_0
    const double inv_norm = 1.0 / norm;
    for (int k = 0; k < kcount; ++k) out[k] *= inv_norm;
}

// one block: points bbox + antennas -> the whole call's range bound and order
// K (the part rule over the whole set: the largest half range over the
// antennas, each about its own centre), and the choice between the Chebyshev
// form and the recurrence (the coefficient tables come per part from
// split_plan_kernel)
__global__ void cheb_plan_kernel(const float* __restrict__ part, int n_part, const float* __restrict__ ant,
                                 int n_ant, double Kd, int n_f, double eps, double k0, ChebPlan* __restrict__ plan) {
    __shared__ float box[6];
    __shared__ float rr[2][256];
    const int t = threadIdx.x;
    if (t < 6) {
        float v = t < 3 ? INFINITY : -INFINITY;
        for (int b = 0; b < n_part; ++b) v = t < 3 ? fminf(v, part[b * 6 + t]) : fmaxf(v, part[b * 6 + t]);
        box[t] = v;
    }
    __syncthreads();
    float hw = 0.0f, ext = 0.0f;
    for (int i = t; i < n_ant; i += blockDim.x) {
        float dn = 0.0f, df = 0.0f;
        for (int d = 0; d < 3; ++d) {
            const float a = ant[d * n_ant + i];
            const float e = fmaxf(fmaxf(box[d] - a, a - box[3 + d]), 0.0f);
            const float f = fmaxf(fabsf(a - box[d]), fabsf(box[3 + d] - a));
            dn += e * e;
            df += f * f;
            ext = fmaxf(ext, f);
        }
        hw = fmaxf(hw, 0.5f * (sqrtf(df) - sqrtf(dn)));
    }
    rr[0][t] = hw;
    rr[1][t] = ext;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (t < k) {
            rr[0][t] = fmaxf(rr[0][t], rr[0][t + k]);
            rr[1][t] = fmaxf(rr[1][t], rr[1][t + k]);
        }
        __syncthreads();
    }
    if (t == 0) {
        const double dr = fmax((double)rr[0][0] * 1.001 + 1e-6, 1e-5);
        const float inv = (float)(1.0 / dr);
        // largest |a_m|: the bin offset (n_f - 1) / 2 from the band's centre
        const double a_max = 3.14159265358979323846 * (n_f - 1) * Kd / (double)inv;
        double J[CH_KMAX + 8];
        bessel_j(a_max, CH_KMAX + 8, J);
        int K = CH_KMAX + 1;
        double tail = 0.0;
        for (int k = CH_KMAX + 7; k >= 0; --k) {
            tail += 2.0 * fabs(J[k]);
            if (tail > eps) { K = k + 1; break; }
        }
        if (K < 2) K = 2;
        // the split-coordinate range in cycles is exact only for axis
        // differences below 1024 cycles (about 2 m at 79 GHz)
        const int direct = K > CH_KMAX || !(rr[1][0] * (float)k0 < kCycAxisMax);
        if (K > CH_KMAX) K = CH_KMAX;
        plan->inv_dr = inv;
        plan->K = K;
        plan->use_direct = direct;
        plan->run_cheb = !direct;
        for (int d = 0; d < 6; ++d) plan->box[d] = box[d];
    }
}

// --------------------------------------------------- spatial order of points
// The Chebyshev parts are runs of consecutive point records; so that a run is
// a compact brick of space rather than a slab of the whole volume, the
// Chebyshev calls pack the points in brick order: the points' bounding box cut
// into 8 x 8 x 8 bricks numbered along a Hilbert curve (a run that ends in one
// brick continues in a face neighbour), a stable counting sort by brick
// (order of the caller kept inside a brick, so the result is deterministic). perm[r] = the point held by record r. Each warp owns a
// sub-chunk of PO_SUB consecutive points: histogram per sub-chunk, exclusive
// scan over sub-chunks in segments of PO_SEG and over the segments and the
// buckets, then each warp places its points in order (peers of equal bucket
// ranked by lane within each round of 32).
constexpr int PO_BUCKETS = 512;
constexpr int PO_SUB = 512;
constexpr int PO_WARPS = 16;
constexpr int PO_SEG = 64;

// Index of brick (x, y, z), 3 bits per axis, along a 3-D Hilbert curve
// (Skilling's transpose form, AIP Conf. Proc. 707, 2004): undo the excess
// work of the inverse transform bit plane by bit plane, Gray-encode, then
// read the index bits out plane-major. Consecutive indices are face
// neighbours, so a run of records that straddles two bricks stays compact.
__device__ __forceinline__ int hilbert_brick(int x, int y, int z) {
    int X[3] = {x, y, z};
#pragma unroll
    for (int Q = 4; Q > 1; Q >>= 1) {
        const int P = Q - 1;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            if (X[i] & Q) {
                X[0] ^= P;
            } else {
                const int t = (X[0] ^ X[i]) & P;
                X[0] ^= t;
                X[i] ^= t;
            }
        }
    }
    X[1] ^= X[0];
    X[2] ^= X[1];
    int t = 0;
#pragma unroll
    for (int Q = 4; Q > 1; Q >>= 1)
        if (X[2] & Q) t ^= Q - 1;
    X[0] ^= t;
    X[1] ^= t;
    X[2] ^= t;
    int h = 0;
#pragma unroll
    for (int j = 2; j >= 0; --j)
        h = (h << 3) | (((X[0] >> j) & 1) << 2) | (((X[1] >> j) & 1) << 1) | ((X[2] >> j) & 1);
    return h;
}

__device__ __forceinline__ int point_bucket(float x, float y, float z, const float (&box)[6]) {
    const float v[3] = {x, y, z};
    int b[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        const float span = box[3 + d] - box[d];
        const int c = span > 0.0f ? (int)((v[d] - box[d]) * (8.0f / span)) : 0;
        b[d] = min(max(c, 0), 7);
    }
    return hilbert_brick(b[0], b[1], b[2]);
}

__global__ void __launch_bounds__(32 * PO_WARPS) point_hist_kernel(const float* __restrict__ xyz, int64_t n,
                                                                   const ChebPlan* __restrict__ plan,
                                                                   uint16_t* __restrict__ bkt,
                                                                   int* __restrict__ hist) {
    __shared__ int h[PO_WARPS][PO_BUCKETS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int i = lane; i < PO_BUCKETS; i += 32) h[warp][i] = 0;
    __syncwarp();
    float box[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) box[d] = plan->box[d];
    const int64_t sc = (int64_t)blockIdx.x * PO_WARPS + warp;
    const int64_t j0 = sc * PO_SUB, j1 = min(n, j0 + PO_SUB);
    for (int64_t j = j0 + lane; j < j1; j += 32) {
        const int b = point_bucket(xyz[j], xyz[n + j], xyz[2 * n + j], box);
        bkt[j] = (uint16_t)b;
        atomicAdd(&h[warp][b], 1);
    }
    __syncwarp();
    for (int i = lane; i < PO_BUCKETS; i += 32) hist[sc * PO_BUCKETS + i] = h[warp][i];
}

// exclusive scan over the sub-chunks of one segment, per bucket, in place;
// seg[segment][bucket] = the segment's totals
__global__ void point_scan_segments(int* __restrict__ hist, int64_t n_sub, int* __restrict__ seg) {
    const int b = threadIdx.x;
    const int64_t s0 = (int64_t)blockIdx.x * PO_SEG, s1 = min(n_sub, s0 + PO_SEG);
    int run = 0;
    for (int64_t sc = s0; sc < s1; ++sc) {
        const int v = hist[sc * PO_BUCKETS + b];
        hist[sc * PO_BUCKETS + b] = run;
        run += v;
    }
    seg[(int64_t)blockIdx.x * PO_BUCKETS + b] = run;
}

// exclusive scan over the segments per bucket (in place), then over the
// buckets: base[b] = the number of points in buckets below b
__global__ void point_scan_totals(int* __restrict__ seg, int n_seg, int* __restrict__ base) {
    __shared__ int tot[PO_BUCKETS];
    const int b = threadIdx.x;
    int run = 0;
    for (int g = 0; g < n_seg; ++g) {
        const int v = seg[(int64_t)g * PO_BUCKETS + b];
        seg[(int64_t)g * PO_BUCKETS + b] = run;
        run += v;
    }
    tot[b] = run;
    __syncthreads();
    if (b == 0) {
        int acc = 0;
        for (int i = 0; i < PO_BUCKETS; ++i) {
            const int v = tot[i];
            tot[i] = acc;
            acc += v;
        }
    }
    __syncthreads();
    base[b] = tot[b];
}

__global__ void __launch_bounds__(32 * PO_WARPS) point_scatter_kernel(const uint16_t* __restrict__ bkt, int64_t n,
                                                                      const int* __restrict__ hist,
                                                                      const int* __restrict__ seg,
                                                                      const int* __restrict__ base,
                                                                      int* __restrict__ perm) {
    __shared__ int cnt[PO_WARPS][PO_BUCKETS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t sc = (int64_t)blockIdx.x * PO_WARPS + warp;
    const int64_t g = sc / PO_SEG;
    for (int i = lane; i < PO_BUCKETS; i += 32)
        cnt[warp][i] = base[i] + seg[g * PO_BUCKETS + i] + hist[sc * PO_BUCKETS + i];
    __syncwarp();
    const int64_t j0 = sc * PO_SUB, j1 = min(n, j0 + PO_SUB);
    for (int64_t jb = j0; jb < j1; jb += 32) {
        const int64_t j = jb + lane;
        const unsigned active = __ballot_sync(0xffffffffu, j < j1);
        if (j < j1) {
            const int b = bkt[j];
            const unsigned peers = __match_any_sync(active, b);
            const int rank = __popc(peers & ((1u << lane) - 1u));
            perm[cnt[warp][b] + rank] = (int)j;
            __syncwarp(active);
            if (rank == 0) cnt[warp][b] += __popc(peers);
        }
        __syncwarp();
    }
}

// records' source order -> permuted SoA copy of three coordinate planes
__global__ void gather_xyz(const float* __restrict__ xyz, int64_t n, const int* __restrict__ perm,
                           float* __restrict__ out) {
    const int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (r >= n) return;
    const int64_t j = perm[r];
    out[r] = xyz[j];
    out[n + r] = xyz[n + j];
    out[2 * n + r] = xyz[2 * n + j];
}

// Expansion of one part of a Chebyshev call (a split of point tiles, possibly
// times a block of antennas, for the to-bins sums; a group of points for the
// to-points sums): its half range 1/inv_dr (each antenna's interval is centred
// on that antenna's own range centre, rcs) and order K.
struct SplitPlan {
    float inv_dr;
    int K;
};

struct ChebBinsArgs {
    const PtRec* pts;          // tiles of CH_TP records
    const float4* ant;         // n_ant_pad (x, y, z, c_ant)
    int n_ant;
    int n_tiles;
    int tiles_per_split;
    const ChebPlan* plan;      // the whole call's plan (run_cheb)
    const SplitPlan* splan;    // [splits][plan_blocks]
    int plan_blocks;           // antenna blocks with their own plan: 1 or gridDim.x
    const float* rcs;          // [splits][n_rec]: each antenna record's range centre (cycles)
    int n_rec;
    const int* kmax;           // largest part order: picks the kernel instance
    double k0;                 // K0 = 2 f_c / c at the band centre f_c, cycles per metre (positions in cycles)
    float amp_scale;           // factor of every moment: gamma's 1 / (16 pi^2) per square cycle (render), 1
    float2* partial;           // [splits][n_ant][CH_KMAX]
    int* err;
};

// thread = antenna: Chebyshev moments of the antenna over the split's points.
// Inner sums over CH_FLUSH tiles in registers, outer FP32 sums in shared memory.
// The core is 3 scalar FMAs per order (T_k recurrence, real and imaginary
// accumulation): the FMA pipe, not the issue rate, bounds this kernel, and a
// packed (re, im) form would spend a wasted lane on the recurrence.
// KC = 8-order groups held in registers: the KC = 3 and KC = 4 instances run
// when the largest part order is at most 24 or 32, each CTA with its part's
// order rounded up to even (at least 8) as a compile-time loop bound (one
// unrolled tile body per even order); the KC = 8 instance (orders beyond 32
// guarded by the part's K) otherwise; all are launched and those that do not
// apply return at once. Each part = (split of points, block of CH_THREADS
// antennas) expands the bin phase over its own half range (SplitPlan), each
// antenna about its own range centre (rcs).
// This thread's antenna for the to-bins tiles, every value in both lanes:
// split position in cycles (h, l), c_ant, and its range centre for the part.
struct BinsAnt {
    f2 hx, hy, hz, lx, ly, lz, cw, rc;
};

// One tile of CH_TP point records (pair layout) against this thread's
// antenna, two points at a time in the two lanes of every packed (f32x2)
// operation: the pair ranges in double-single (the split-coordinate form of
// pair_range_split, lane-wise), amplitude times carrier phasor, and the
// moments M'_k += A V_k for k < KE (KE even, fixed at compile time), V_k =
// s_k T_k(x) with s_k = (-1)^floor(k/2) by the sign-alternating recurrence
// V_k = (-/+ 2x) V_{k-1} + V_{k-2} (minus for even k), one packed FMA for both
// points; the moments themselves are scalar sums over both lanes, and s_k is
// applied when they are written. Only the square roots, the sincos and the
// rounding and clamps run per lane. kGuard (the 64-order instance): orders
// past 32 run in blocks of 8 up to the part's own order K.
template <bool kComplexAmp, int KM, int KE, bool kGuard>
__device__ __forceinline__ void bins_tile(const float4* __restrict__ tile, const BinsAnt& A, f2 INV, f2 HINV, int K,
                                          float (&mr)[KM], float (&mi)[KM]) {
    const f2 TWO = pk2(2.0f, 2.0f), NEG1 = pk2(-1.0f, -1.0f), HALF = pk2(0.5f, 0.5f);
#pragma unroll kBinsUnroll
    for (int p = 0; p < CH_TP / 2; ++p) {
        const ulonglong2* Q = reinterpret_cast<const ulonglong2*>(tile + 6 * p);
        // fields in pairs: (xh | yh), (zh | w or c_re), (n'x or c_im | n'y), (n'z | t_eff), (xl | yl), (zl | e)
        const ulonglong2 q0 = Q[0], q1 = Q[1], q2 = Q[2], q4 = Q[4], q5 = Q[5];
        const f2 hx = sub2(q0.x, A.hx), hy = sub2(q0.y, A.hy), hz = sub2(q1.x, A.hz);
        const f2 lx = sub2(q4.x, A.lx), ly = sub2(q4.y, A.ly), lz = sub2(q5.x, A.lz);
        const f2 Sh = fma2(hz, hz, fma2(hy, hy, mul2(hx, hx)));              // exact
        const f2 cross = fma2(lx, fma2(TWO, hx, lx), fma2(ly, fma2(TWO, hy, ly), mul2(lz, fma2(TWO, hz, lz))));
        float s0, s1;
        upk2(add2(Sh, cross), s0, s1);
        s0 = fmaxf(s0, 1e-30f);
        s1 = fmaxf(s1, 1e-30f);
        const f2 S = pk2(s0, s1), RS = pk2(rsqrtf(s0), rsqrtf(s1));
        const f2 r0 = mul2(S, RS);
        const f2 rl2 = mul2(add2(fma2(r0, mul2(r0, NEG1), Sh), cross), RS);    // 2 rl: r = r0 + rl
        // carrier phase: the fractional cycle of r0 + rl
        float a0, a1;
        upk2(r0, a0, a1);
        const f2 fr = fma2(rl2, HALF, sub2(r0, pk2(rintf(a0), rintf(a1))));
        f2 AR, AI;
        if (!kComplexAmp) {
            // A / (gamma's constant) = w T'^2 D / r^2: with n' = sqrt2 n,
            // nd = n'.d / r and D = max(nd^2 - e, 0); u = T' / r;
            // A exp(-j 2 pi K0 r) from the sincos of the negated angle
            float f0, f1;
            upk2(mul2(fr, pk2(-6.28318530717958648f, -6.28318530717958648f)), f0, f1);
            float sn0, cs0, sn1, cs1;
            __sincosf(f0, &sn0, &cs0);
            __sincosf(f1, &sn1, &cs1);
            const ulonglong2 q3 = Q[3];
            const f2 dx = add2(hx, lx), dy = add2(hy, ly), dz = add2(hz, lz);
            const f2 nd = mul2(fma2(q3.x, dz, fma2(q2.y, dy, mul2(q2.x, dx))), RS);
            float d0, d1, v0, v1;
            upk2(fma2(nd, nd, q5.y), d0, d1);                                // nd^2 - e (records hold -e)
            upk2(sub2(q3.y, A.cw), v0, v1);
            const f2 D = pk2(fmaxf(d0, 0.0f), fmaxf(d1, 0.0f));
            const f2 u = mul2(pk2(__saturatef(v0), __saturatef(v1)), RS);
            const f2 amp = mul2(q1.y, mul2(mul2(u, u), D));
            AR = mul2(amp, pk2(cs0, cs1));
            AI = mul2(amp, pk2(sn0, sn1));
        } else {
            float f0, f1;
            upk2(mul2(fr, pk2(6.28318530717958648f, 6.28318530717958648f)), f0, f1);
            float sn0, cs0, sn1, cs1;
            __sincosf(f0, &sn0, &cs0);
            __sincosf(f1, &sn1, &cs1);
            const f2 CS = pk2(cs0, cs1), SN = pk2(sn0, sn1);
            const f2 cr = q1.y, ci = q2.x;
            AR = fma2(ci, SN, mul2(cr, CS));                                 // c exp(-j 2 pi K0 r)
            AI = fma2(cr, mul2(SN, NEG1), mul2(ci, CS));
        }
        const f2 xs = fma2(rl2, HINV, mul2(sub2(r0, A.rc), INV));             // (r - r_c) / dr
        float ar0, ar1, ai0, ai1, x0, x1;
        upk2(AR, ar0, ar1);
        upk2(AI, ai0, ai1);
        upk2(xs, x0, x1);
        mr[0] += ar0 + ar1;
        mi[0] += ai0 + ai1;
        mr[1] = fmaf(ar0, x0, fmaf(ar1, x1, mr[1]));
        mi[1] = fmaf(ai0, x0, fmaf(ai1, x1, mi[1]));
        const f2 mp = mul2(TWO, xs), mn = mul2(pk2(-2.0f, -2.0f), xs);
        f2 vkm1 = pk2(1.0f, 1.0f), vk = xs;                                  // V_0, V_1
#pragma unroll
        for (int kc = 0; kc < KE; kc += 8) {
            if (!kGuard || kc < 32 || kc < K) {
#pragma unroll
                for (int kk = 0; kk < 8; ++kk) {
                    const int k = kc + kk;
                    if (k >= 2 && k < KE) {
                        const f2 vn = fma2((k & 1) ? mp : mn, vk, vkm1);
                        vkm1 = vk;
                        vk = vn;
                        float w0, w1;
                        upk2(vn, w0, w1);
                        mr[k] = fmaf(ar0, w0, fmaf(ar1, w1, mr[k]));
                        mi[k] = fmaf(ai0, w0, fmaf(ai1, w1, mi[k]));
                    }
                }
            }
        }
    }
}

#define GERAF_BINS_CASE(E) \
    case E: bins_tile<kComplexAmp, KM, ((E) < KM ? (E) : KM), false>(tile, BA, INV, HINV, K, mr, mi); break;

template <bool kComplexAmp, int KC>
__global__ void __launch_bounds__(CH_THREADS, (KC == 3 && !kComplexAmp) ? GERAF_CH_BINS_CTAS_24
                                                                     : (KC <= 4 ? GERAF_CH_BINS_CTAS : 1))
    cheb_bins_kernel(const ChebBinsArgs args) {
    constexpr int KM = 8 * KC;
    constexpr int KU = KC < 4 ? 8 * KC : 32;                 // orders every flush covers
    if (!args.plan->run_cheb) return;
    {
        const int km = *args.kmax;
        const int want = km <= 24 ? 3 : (km <= 32 ? 4 : 8);
        if (want != KC) return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    PtRec* tiles = reinterpret_cast<PtRec*>(smem);                              // [2][CH_TP]
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem + 2 * CH_TP * sizeof(PtRec));
    int* abort_flag = reinterpret_cast<int*>(bar + 2);
    float2* outer = reinterpret_cast<float2*>(smem + 2 * CH_TP * sizeof(PtRec) + 32);   // [KM][CH_THREADS]
    const int t = threadIdx.x;
    const int ia = blockIdx.x * CH_THREADS + t;
    const int split = blockIdx.y;
    const int tile0 = split * args.tiles_per_split;
    const int tile1 = min(tile0 + args.tiles_per_split, args.n_tiles);
    const int n_my = tile1 - tile0;
    const SplitPlan sp = args.splan[split * args.plan_blocks + (args.plan_blocks > 1 ? blockIdx.x : 0)];
    const int K = sp.K;
    const int ke = K <= 8 ? 8 : (K + 1) & ~1;                // orders run: K rounded up to even, >= 8
    const f2 INV = pk2(sp.inv_dr, sp.inv_dr), HINV = pk2(0.5f * sp.inv_dr, 0.5f * sp.inv_dr);
    const float r_c = args.rcs[(size_t)split * args.n_rec + ia];   // this antenna's range centre
    const float4 A4 = args.ant[ia];                          // padded: always readable
    BinsAnt BA;
    {
        float4 Ah, Al;
        split3c(A4.x, A4.y, A4.z, args.k0, Ah, Al);
        BA.hx = pk2(Ah.x, Ah.x); BA.hy = pk2(Ah.y, Ah.y); BA.hz = pk2(Ah.z, Ah.z);
        BA.lx = pk2(Al.x, Al.x); BA.ly = pk2(Al.y, Al.y); BA.lz = pk2(Al.z, Al.z);
        BA.cw = pk2(A4.w, A4.w); BA.rc = pk2(r_c, r_c);
    }
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    for (int k = 0; k < KM; ++k) outer[k * CH_THREADS + t] = make_float2(0.0f, 0.0f);
    __syncthreads();
    const uint32_t tile_bytes = (uint32_t)(CH_TP * sizeof(PtRec));
    if (t == 0)
        for (int s = 0; s < 2 && s < n_my; ++s) {
            mbar_arrive_expect_tx(&bar[s], tile_bytes);
            tma_load_1d(tiles + s * CH_TP, args.pts + (size_t)(tile0 + s) * CH_TP, tile_bytes, &bar[s]);
        }
    float mr[KM], mi[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) mr[k] = mi[k] = 0.0f;

    for (int it = 0; it < n_my; ++it) {
        const int buf = it & 1;
        if (!mbar_wait(&bar[buf], (it >> 1) & 1)) atomicOr(abort_flag, 1);
        __syncthreads();
        if (*abort_flag) {
            if (t == 0) {
                atomicOr(args.err, 1);
                mbar_drain2(bar, it, n_my);
            }
            return;
        }
        const float4* tile = reinterpret_cast<const float4*>(tiles + buf * CH_TP);
        if constexpr (KC == 8) {
            bins_tile<kComplexAmp, KM, KM, true>(tile, BA, INV, HINV, K, mr, mi);
        } else {
            switch (ke) {
                GERAF_BINS_CASE(8) GERAF_BINS_CASE(10) GERAF_BINS_CASE(12) GERAF_BINS_CASE(14)
                GERAF_BINS_CASE(16) GERAF_BINS_CASE(18) GERAF_BINS_CASE(20) GERAF_BINS_CASE(22)
                GERAF_BINS_CASE(24) GERAF_BINS_CASE(26) GERAF_BINS_CASE(28) GERAF_BINS_CASE(30)
                default: bins_tile<kComplexAmp, KM, KM, false>(tile, BA, INV, HINV, K, mr, mi);
            }
        }
        if (((it + 1) % CH_FLUSH) == 0 || it + 1 == n_my) {
#pragma unroll
            for (int kc = 0; kc < KM; kc += 8)
                if (kc < KU || kc < K)
#pragma unroll
                    for (int kk = 0; kk < 8; ++kk) {
                        float2 o = outer[(kc + kk) * CH_THREADS + t];
                        o.x += mr[kc + kk];
                        o.y += mi[kc + kk];
                        outer[(kc + kk) * CH_THREADS + t] = o;
                        mr[kc + kk] = mi[kc + kk] = 0.0f;
                    }
        }
        __syncthreads();
        if (t == 0 && it + 2 < n_my) {
            mbar_arrive_expect_tx(&bar[buf], tile_bytes);
            tma_load_1d(tiles + buf * CH_TP, args.pts + (size_t)(tile0 + it + 2) * CH_TP, tile_bytes, &bar[buf]);
        }
    }
    if (ia < args.n_ant) {
        // M_k = s_k M'_k, s_k = (-1)^floor(k/2)
        float2* dst = args.partial + ((size_t)split * args.n_ant + ia) * CH_KMAX;
        for (int k = 0; k < K; ++k) {
            const float2 o = outer[k * CH_THREADS + t];
            const float sc = ((k >> 1) & 1) ? -args.amp_scale : args.amp_scale;
            dst[k] = make_float2(o.x * sc, o.y * sc);
        }
    }
}

// bounding box of each split's records (pair layout; positions rebuilt exactly
// as xh + xl; padding records included, they sit at a real point's position)
__global__ void split_bbox_kernel(const PtRec* __restrict__ pts, int n_tiles, int tiles_per_split,
                                  float* __restrict__ box) {
    __shared__ float red[6][256];
    const int sp = blockIdx.x;
    const int64_t r0 = (int64_t)sp * tiles_per_split * CH_TP;
    const int64_t r1 = min((int64_t)(sp + 1) * tiles_per_split, (int64_t)n_tiles) * CH_TP;
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        // the pair layout: (xh, yh, zh) are fields 0-2, (xl, yl, zl) fields 8-10
        const float x[3] = {pair_field(pts, r, 0) + pair_field(pts, r, 8), pair_field(pts, r, 1) + pair_field(pts, r, 9),
                            pair_field(pts, r, 2) + pair_field(pts, r, 10)};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            mn[d] = fminf(mn[d], x[d]);
            mx[d] = fmaxf(mx[d], x[d]);
        }
    }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        red[d][threadIdx.x] = mn[d];
        red[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k)
            for (int d = 0; d < 3; ++d) {
                red[d][threadIdx.x] = fminf(red[d][threadIdx.x], red[d][threadIdx.x + k]);
                red[3 + d][threadIdx.x] = fmaxf(red[3 + d][threadIdx.x], red[3 + d][threadIdx.x + k]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) box[sp * 6 + threadIdx.x] = red[threadIdx.x][0];
}

// One block per part = (split or group of points sp, block of antennas b),
// parts in order sp * n_ab + b (n_ab blocks of ant_per_block consecutive
// antenna records in the spatial order, or one block of all antennas): each
// record's range centre r_c(i) (midpoint of its nearest and farthest range to
// the points' box, written to rcs[sp][i] for every record, padding ones
// included), the part's half range (the largest over its antennas of half
// that span), its order K (the whole call's rule: Bessel tail <= eps) and its
// FP32 coefficient table Cs[part][k][n] = eps_k (-j)^k J_k(a_m), m = n -
// (n_f - 1) / 2. kmax collects the largest part order.
// Double-single FP32 arithmetic (value = h + l, |l| <= ulp(h) / 2) for the
// coefficient tables: error-free products by FMA and Knuth's two-sum, so the
// Bessel recurrence keeps ~44 bits without FP64 (slow on this part).
struct DS {
    float h, l;
};
__device__ __forceinline__ DS ds_renorm(float s, float e) {
    const float h = __fadd_rn(s, e);
    return DS{h, __fsub_rn(e, __fsub_rn(h, s))};
}
__device__ __forceinline__ DS ds_mul(DS a, DS b) {
    const float p = __fmul_rn(a.h, b.h);
    float e = __fmaf_rn(a.h, b.h, -p);
    e = __fmaf_rn(a.h, b.l, e);
    e = __fmaf_rn(a.l, b.h, e);
    return ds_renorm(p, e);
}
__device__ __forceinline__ DS ds_mulf(DS a, float b) {
    const float p = __fmul_rn(a.h, b);
    float e = __fmaf_rn(a.h, b, -p);
    e = __fmaf_rn(a.l, b, e);
    return ds_renorm(p, e);
}
__device__ __forceinline__ DS ds_add(DS a, DS b) {
    const float s = __fadd_rn(a.h, b.h);
    const float bb = __fsub_rn(s, a.h);
    float e = __fadd_rn(__fsub_rn(a.h, __fsub_rn(s, bb)), __fsub_rn(b.h, bb));
    e = __fadd_rn(e, __fadd_rn(a.l, b.l));
    return ds_renorm(s, e);
}

// C[k n_f] for k < K, one bin: (2 - [k = 0]) J_k(s a) (-j)^k for a >= 0 and
// the sign s = -1 when neg (J_k(-a) = (-1)^k J_k(a), so the factor becomes
// j^k), J_k by Miller's backward recurrence in double-single, normalised by
// J_0 + 2 sum J_2m = 1. Two passes over the same recurrence: the first finds
// the normalisation and how often the running values were rescaled (by
// 1e-20 whenever they pass 1e20), the second writes each J_k scaled into the
// final scale (a value recorded two or more rescales before the end is below
// 1e-20 of the largest and written as 0).
// 2 / a in double-single: the FP32 quotient and one correction by the residual
__device__ __forceinline__ DS ds_two_over(DS a) {
    const float r0 = __fdiv_rn(2.0f, a.h);
    const float p = __fmul_rn(a.h, r0);
    const float pe = __fmaf_rn(a.h, r0, -p);
    float e = __fsub_rn(2.0f, p);            // exact: p is within an ulp of 2
    e = __fsub_rn(e, pe);
    e = __fmaf_rn(-a.l, r0, e);
    return ds_renorm(r0, __fmul_rn(e, __fmul_rn(0.5f, r0)));   // 2/a = r0 + e r0 / 2 to second order
}

__device__ void bessel_table_ds(DS a, int K, bool neg, float2* __restrict__ C, int n_f) {
    if (!(a.h > 1e-20f)) {                   // J_0 = 1, the others vanish
        for (int k = 0; k < K; ++k) C[(size_t)k * n_f] = make_float2(k == 0 ? 1.0f : 0.0f, 0.0f);
        return;
    }
    int start = K + 20 + (int)a.h;
    start += start & 1;
    const DS inv2 = ds_two_over(a);
    int R = 0;
    DS nrm{0.0f, 0.0f};
    for (int pass = 0; pass < 2; ++pass) {
        DS jp1{0.0f, 0.0f}, j{1e-30f, 0.0f};
        DS acc{0.0f, 0.0f};
        int r = 0;
        float inv_n = 0.0f;
        if (pass == 1) inv_n = (float)(1.0 / ((double)nrm.h + (double)nrm.l));
        for (int k = start; k >= 1; --k) {
            const DS jm1 = ds_add(ds_mul(ds_mulf(inv2, (float)k), j), DS{-jp1.h, -jp1.l});
            jp1 = j;
            j = jm1;
            if (fabsf(j.h) > 1e20f) {
                j = ds_mulf(j, 1e-20f);
                jp1 = ds_mulf(jp1, 1e-20f);
                acc = ds_mulf(acc, 1e-20f);
                ++r;
            }
            const int q = k - 1;
            if (pass == 0) {
                if ((q & 1) == 0 && q > 0) acc = ds_add(acc, ds_mulf(j, 2.0f));
            } else if (q < K) {
                const int lag = R - r;
                float v = lag >= 2 ? 0.0f : __fadd_rn(j.h, j.l) * inv_n;
                if (lag == 1) v *= 1e-20f;
                const float m = q == 0 ? v : 2.0f * v;
                // m (-j)^q, or m j^q for a negative argument
                const float si = neg ? -m : m;
                float2 c;
                switch (q & 3) {
                    case 0: c = make_float2(m, 0.0f); break;
                    case 1: c = make_float2(0.0f, -si); break;
                    case 2: c = make_float2(-m, 0.0f); break;
                    default: c = make_float2(0.0f, si); break;
                }
                C[(size_t)q * n_f] = c;
            }
        }
        if (pass == 0) {
            nrm = ds_add(acc, j);                // + J_0
            R = r;
        }
    }
}

// The expansion order for argument a: the smallest K with
// sum_{k >= K} 2 |J_k(a)| <= eps over k < kcount (K >= 1), by the same two-pass
// double-single recurrence: the first pass normalises, the second accumulates
// the tail from the top and stops where it first exceeds eps.
__device__ int bessel_order_ds(DS a, int kcount, float eps) {
    if (!(a.h > 1e-20f)) return 1;
    int start = kcount + 20 + (int)a.h;
    start += start & 1;
    const DS inv2 = ds_two_over(a);
    int R = 0;
    DS nrm{0.0f, 0.0f};
    for (int pass = 0; pass < 2; ++pass) {
        DS jp1{0.0f, 0.0f}, j{1e-30f, 0.0f};
        DS acc{0.0f, 0.0f};
        float tail = 0.0f;
        int r = 0;
        float inv_n = 0.0f;
        if (pass == 1) inv_n = __fdiv_rn(1.0f, __fadd_rn(nrm.h, nrm.l));
        for (int k = start; k >= 1; --k) {
            const DS jm1 = ds_add(ds_mul(ds_mulf(inv2, (float)k), j), DS{-jp1.h, -jp1.l});
            jp1 = j;
            j = jm1;
            if (fabsf(j.h) > 1e20f) {
                j = ds_mulf(j, 1e-20f);
                jp1 = ds_mulf(jp1, 1e-20f);
                acc = ds_mulf(acc, 1e-20f);
                tail *= 1e-20f;
                ++r;
            }
            const int q = k - 1;
            if (pass == 0) {
                if ((q & 1) == 0 && q > 0) acc = ds_add(acc, ds_mulf(j, 2.0f));
            } else if (q < kcount) {
                tail += 2.0f * fabsf(__fadd_rn(j.h, j.l));
                const int lag = R - r;
                if (lag <= 1) {
                    const float v = tail * inv_n * (lag == 1 ? 1e-20f : 1.0f);
                    if (v > eps) return q + 1;
                }
            }
        }
        if (pass == 0) {
            nrm = ds_add(acc, j);
            R = r;
        }
    }
    return 1;
}

// exp(-j 2 pi m Kc r_c) for the bin offset m (exact in FP32) and the range
// centre r_c in cycles, Kc = kch + kcl in double-single: the fractional cycle
// of m Kc r_c in double-single (error-free products by FMA, so a phase of tens
// of cycles keeps ~1e-12 cycle), then sincospi of its leading part with a
// first-order correction for the rest.
__device__ __forceinline__ float2 bin_phase(float m, float kch, float kcl, float rc) {
    const float p1 = __fmul_rn(kch, rc);
    const DS ph = ds_renorm(p1, __fmaf_rn(kcl, rc, __fmaf_rn(kch, rc, -p1)));
    const float p = __fmul_rn(m, ph.h);
    const float pe = __fmaf_rn(m, ph.h, -p);
    const float t0 = __fsub_rn(p, rintf(p));            // exact
    const float u = __fmaf_rn(m, ph.l, pe);
    const float fh = __fadd_rn(t0, u);
    const float fl = __fsub_rn(u, __fsub_rn(fh, t0));
    float sn, cs;
    sincospif(-2.0f * fh, &sn, &cs);
    const float d = -6.28318530717958648f * fl;          // exp(-j 2 pi fl) = 1 + j d to first order
    return make_float2(__fmaf_rn(-sn, d, cs), __fmaf_rn(cs, d, sn));
}

__global__ void split_plan_kernel(const float* __restrict__ box, const float4* __restrict__ ant, int n_ant,
                                  int n_rec, int n_ab, int ant_per_block, double Kd, int n_f, double eps,
                                  double k0, const ChebPlan* __restrict__ gplan, SplitPlan* __restrict__ splan,
                                  float* __restrict__ rcs, float2* __restrict__ Cs, int* __restrict__ kmax) {
    if (!gplan->run_cheb) return;
    __shared__ float rr[256];
    __shared__ int sK;
    __shared__ DS s_a1;
    const int sp = blockIdx.x, t = threadIdx.x;
    const int b = sp % n_ab;
    const float* bx = box + (sp / n_ab) * 6;     // in cycles
    const int i0 = b * ant_per_block, i1 = min(n_ant, i0 + ant_per_block);
    const int iw = n_ab > 1 ? min(n_rec, i0 + ant_per_block) : n_rec;   // records whose centre this part writes
    float* rc_out = rcs + (size_t)(sp / n_ab) * n_rec;
    const float k0f = (float)k0;
    float hw = 0.0f;
    for (int i = i0 + t; i < iw; i += blockDim.x) {
        float dn = 0.0f, df = 0.0f;
        const float4 A = ant[i];                  // metres
        for (int d = 0; d < 3; ++d) {
            const float a = k0f * (d == 0 ? A.x : (d == 1 ? A.y : A.z));
            const float e = fmaxf(fmaxf(bx[d] - a, a - bx[3 + d]), 0.0f);
            const float f = fmaxf(fabsf(a - bx[d]), fabsf(bx[3 + d] - a));
            dn += e * e;
            df += f * f;
        }
        const float lo = sqrtf(dn), hi = sqrtf(df);
        rc_out[i] = 0.5f * (lo + hi);
        if (i < i1) hw = fmaxf(hw, 0.5f * (hi - lo));
    }
    rr[t] = hw;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (t < k) rr[t] = fmaxf(rr[t], rr[t + k]);
        __syncthreads();
    }
    // the part's half range and table in cycles: Kc = bin phase step in
    // cycles per cycle of range; margins 1e-6 m and 1e-5 m in cycles
    const double Kc = Kd / k0;
    if (t == 0) {
        const double dr = fmax((double)rr[0] * 1.001 + 1e-6 * k0, 1e-5 * k0);
        const float inv = (float)(1.0 / dr);
        // argument step a1 = 2 pi Kc dr per bin of offset (double-single);
        // every bin's argument follows in FP32 arithmetic
        const double dr_f = 1.0 / (double)inv;
        const double a1 = 2.0 * 3.14159265358979323846 * Kc * dr_f;
        const double a_max = a1 * 0.5 * (double)(n_f - 1);
        const DS am{(float)a_max, (float)(a_max - (double)(float)a_max)};
        int K = bessel_order_ds(am, CH_KMAX + 8, (float)eps);
        if (K < 2) K = 2;
        if (K > CH_KMAX) K = CH_KMAX;
        splan[sp] = SplitPlan{inv, K};
        atomicMax(kmax, K);
        sK = K;
        s_a1 = DS{(float)a1, (float)(a1 - (double)(float)a1)};
    }
    __syncthreads();
    const int K = sK;
    const DS a1 = s_a1;
    const float nc = 0.5f * (float)(n_f - 1);
    float2* C = Cs + (size_t)sp * CH_KMAX * n_f;
    for (int n = t; n < n_f; n += blockDim.x) {
        const float m = (float)n - nc;                   // exact: a multiple of 1/2
        bessel_table_ds(ds_mulf(a1, fabsf(m)), K, m < 0.0f, C + n, n_f);
    }
}

// sum over the splits of a group of RS splits of
//   exp(-j 2 pi m Kc r_c(sp, i)) sum_k Cs[sp, b(i)][k][n] M_k(sp, i),
// i an antenna record, b(i) its block of CH_THREADS records, written to the
// antenna the record holds:
// block = (RA antennas, split group); thread = bin, the RA antennas in
// registers so each table value is loaded once; the per-split sums (FP32, at
// most 64 terms) are turned by the record's bin phase and added with Kahan
// compensation across the group's splits.
// The groups' sums are added in FP64, in group order, by sum_split_groups.
constexpr int RA = 4;
constexpr int RS = 32;
static_assert(CH_THREADS % RA == 0, "a reconstruction block stays in one antenna block");
__global__ void cheb_reconstruct_split_kernel(const float2* __restrict__ partial, int splits, int n_ant, int n_f,
                                              int n_ab, const ChebPlan* __restrict__ gplan,
                                              const SplitPlan* __restrict__ splan, const float2* __restrict__ Cs,
                                              const float* __restrict__ rcs, int n_rec, double kc,
                                              const int* __restrict__ perm, float2* __restrict__ group_out) {
    if (!gplan->run_cheb) return;
    const int i0 = blockIdx.x * RA;
    const int b = n_ab > 1 ? i0 / CH_THREADS : 0;   // antenna block of all RA antennas (RA divides CH_THREADS)
    const int s0 = blockIdx.y * RS, s1 = min(splits, s0 + RS);
    const float kch = (float)kc, kcl = (float)(kc - (double)kch);
    const float nc = 0.5f * (float)(n_f - 1);
    for (int n = threadIdx.x; n < n_f; n += blockDim.x) {
        const float m = (float)n - nc;
        float hr[RA], hi[RA], cr_[RA], ci_[RA];
#pragma unroll
        for (int q = 0; q < RA; ++q) hr[q] = hi[q] = cr_[q] = ci_[q] = 0.0f;
        for (int s = s0; s < s1; ++s) {
            const int part = s * n_ab + b;
            const int K = splan[part].K;
            const float2* C = Cs + (size_t)part * CH_KMAX * n_f + n;
            float sr[RA], si[RA];
#pragma unroll
            for (int q = 0; q < RA; ++q) sr[q] = si[q] = 0.0f;
            for (int k = 0; k < K; ++k) {
                const float2 c = C[(size_t)k * n_f];
#pragma unroll
                for (int q = 0; q < RA; ++q) {
                    const int i = min(i0 + q, n_ant - 1);
                    const float2 mo = partial[((size_t)s * n_ant + i) * CH_KMAX + k];
                    sr[q] = fmaf(c.x, mo.x, fmaf(-c.y, mo.y, sr[q]));
                    si[q] = fmaf(c.x, mo.y, fmaf(c.y, mo.x, si[q]));
                }
            }
#pragma unroll
            for (int q = 0; q < RA; ++q) {
                const float2 ph = bin_phase(m, kch, kcl, rcs[(size_t)s * n_rec + min(i0 + q, n_ant - 1)]);
                const float pr = ph.x * sr[q] - ph.y * si[q], pi = ph.x * si[q] + ph.y * sr[q];
                float y = pr - cr_[q], tt = hr[q] + y;
                cr_[q] = (tt - hr[q]) - y;
                hr[q] = tt;
                y = pi - ci_[q];
                tt = hi[q] + y;
                ci_[q] = (tt - hi[q]) - y;
                hi[q] = tt;
            }
        }
#pragma unroll
        for (int q = 0; q < RA; ++q)
            if (i0 + q < n_ant)     // record i0 + q holds antenna perm[i0 + q]
                group_out[((size_t)blockIdx.y * n_ant + perm[i0 + q]) * n_f + n] = make_float2(hr[q], hi[q]);
    }
}

__global__ void sum_split_groups(const float2* __restrict__ group_out, int groups, int64_t n,
                                 const ChebPlan* __restrict__ gplan, float2* __restrict__ out) {
    if (!gplan->run_cheb) return;
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= n) return;
    double sr = 0.0, si = 0.0;
    for (int g = 0; g < groups; ++g) {
        const float2 v = group_out[(size_t)g * n + e];
        sr += v.x;
        si += v.y;
    }
    out[e] = make_float2((float)sr, (float)si);
}

size_t cheb_bins_smem(int km) { return 2 * CH_TP * sizeof(PtRec) + 32 + (size_t)km * CH_THREADS * sizeof(float2); }

// antenna rows for the Chebyshev point kernels: four heads with every value
// twice, so that one 16-byte load gives two packed (f32x2) operands:
// (xh, xh, yh, yh), (zh, zh, c, c), (xl, xl, yl, yl), (zl, zl, r_c, r_c) (the
// split position, c_ant and the antenna's range centre for the group), then
// CH_KMAX float4 s_k (h_re, h_re, h_im, h_im) with h_k = sum_n sig(n) * (conj ?
// conj(C_k(n)) : C_k(n)), sig = (conj_sig ? conj(v) : v) and s_k =
// (-1)^floor(k/2), the sign of the point kernels' packed V_k = s_k T_k
// recurrence
constexpr int CH_HEADS = 4;
constexpr int CH_ROW = CH_HEADS + CH_KMAX;

// Bounding box of each group of per_group consecutive points (xyz in [3][n]
// layout): box[g] = (min x, min y, min z, max x, max y, max z).
__global__ void group_bbox_kernel(const float* __restrict__ xyz, int64_t n, int64_t per_group, float k0f,
                                  float* __restrict__ box) {
    __shared__ float red[6][256];
    const int g = blockIdx.x;
    const int64_t j0 = (int64_t)g * per_group, j1 = min(n, j0 + per_group);
    float mn[3] = {INFINITY, INFINITY, INFINITY}, mx[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x)
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            const float x = xyz[d * n + j];
            mn[d] = fminf(mn[d], x);
            mx[d] = fmaxf(mx[d], x);
        }
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        red[d][threadIdx.x] = mn[d];
        red[3 + d][threadIdx.x] = mx[d];
    }
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k)
            for (int d = 0; d < 3; ++d) {
                red[d][threadIdx.x] = fminf(red[d][threadIdx.x], red[d][threadIdx.x + k]);
                red[3 + d][threadIdx.x] = fmaxf(red[3 + d][threadIdx.x], red[3 + d][threadIdx.x + k]);
            }
        __syncthreads();
    }
    if (threadIdx.x < 6) box[g * 6 + threadIdx.x] = red[threadIdx.x][0] * k0f;   // cycles (k0f > 0)
}

// Antenna rows of the to-points kernels, one set per point group g: row r
// holds the antenna perm[r] (the spatial order), planned with the part
// (g, b = r / CH_THREADS) when the groups are planned per antenna block (n_ab
// blocks), else with the group's plan over all antennas (n_ab = 1):
// row(g, r) = the heads (the antenna's split position in cycles, c_ant, the
// record's range centre r_c(g, r); CH_ROW), then for
// k < CH_KMAX the packed s_k h_k, h_k = sum_n sig(i, n) P(r, n) C_part,k(n),
// P = exp(-j 2 pi m Kc r_c) the record's bin phase (P and C both conjugated,
// and sig, on request), zero beyond the part's order and for padding antennas.
// Block = GR_T records of one group (inside one antenna block); thread = one
// order k and every fourth record of the tile; bins (turned by their phase)
// staged in shared memory in chunks of GR_NC; FP32 sums.
constexpr int GR_T = 16;
constexpr int GR_NC = 64;
static_assert(CH_THREADS % GR_T == 0, "a rows block stays in one antenna block");
__global__ void __launch_bounds__(256) cheb_group_rows_kernel(
    const float* __restrict__ ant, const float* __restrict__ c_ant, const float2* __restrict__ sig,
    const int* __restrict__ perm, int n_ant, int n_ant_pad, int n_f, int n_ab, const ChebPlan* __restrict__ plan,
    const SplitPlan* __restrict__ gplan, const float2* __restrict__ Cs, const float* __restrict__ rcs, double kc,
    int conj_c, int conj_sig, double k0, float4* __restrict__ rows) {
    if (!plan->run_cheb) return;
    __shared__ float2 sC[CH_KMAX][GR_NC + 1];
    __shared__ float2 sS[GR_T][GR_NC + 1];
    __shared__ float sRc[GR_T];
    const int g = blockIdx.y, i0 = blockIdx.x * GR_T, t = threadIdx.x;
    const int part = g * n_ab + (n_ab > 1 ? i0 / CH_THREADS : 0);
    const int K = gplan[part].K;
    float4* grow = rows + (size_t)g * n_ant_pad * CH_ROW;
    const float* grc = rcs + (size_t)g * n_ant_pad;
    if (t < GR_T) {
        const int i = min(i0 + t, n_ant_pad - 1);
        sRc[t] = grc[i];
        if (i0 + t < n_ant_pad) {
            const int q = i < n_ant ? perm[i] : 0;
            float4 hi, lo;
            split3c(ant[q], ant[n_ant + q], ant[2 * n_ant + q], k0, hi, lo);
            const float cw = c_ant ? c_ant[q] : 0.0f, rc = grc[i];
            float4* h = grow + (size_t)i * CH_ROW;
            h[0] = make_float4(hi.x, hi.x, hi.y, hi.y);
            h[1] = make_float4(hi.z, hi.z, cw, cw);
            h[2] = make_float4(lo.x, lo.x, lo.y, lo.y);
            h[3] = make_float4(lo.z, lo.z, rc, rc);
        }
    }
    const float kch = (float)kc, kcl = (float)(kc - (double)kch);
    const float nc = 0.5f * (float)(n_f - 1);
    const int k = t >> 2, r = t & 3;
    const float2* C = Cs + (size_t)part * CH_KMAX * n_f;
    float ar[4] = {0.0f, 0.0f, 0.0f, 0.0f}, ai[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    for (int n0 = 0; n0 < n_f; n0 += GR_NC) {
        const int nc_ = min(GR_NC, n_f - n0);
        __syncthreads();
        for (int e = t; e < CH_KMAX * GR_NC; e += blockDim.x) {
            const int kk = e / GR_NC, nn = e % GR_NC;
            float2 c = make_float2(0.0f, 0.0f);
            if (kk < K && nn < nc_) {
                c = C[(size_t)kk * n_f + n0 + nn];
                if (conj_c) c.y = -c.y;
            }
            sC[kk][nn] = c;
        }
        for (int e = t; e < GR_T * GR_NC; e += blockDim.x) {
            const int a = e / GR_NC, nn = e % GR_NC, i = i0 + a;
            float2 v = make_float2(0.0f, 0.0f);
            if (i < n_ant && nn < nc_) {
                v = sig[(size_t)perm[i] * n_f + n0 + nn];
                if (conj_sig) v.y = -v.y;
                float2 ph = bin_phase((float)(n0 + nn) - nc, kch, kcl, sRc[a]);
                if (conj_c) ph.y = -ph.y;
                v = make_float2(v.x * ph.x - v.y * ph.y, v.x * ph.y + v.y * ph.x);
            }
            sS[a][nn] = v;
        }
        __syncthreads();
        if (k < K)
            for (int nn = 0; nn < nc_; ++nn) {
                const float2 c = sC[k][nn];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float2 v = sS[r + 4 * q][nn];
                    ar[q] = fmaf(v.x, c.x, fmaf(-v.y, c.y, ar[q]));
                    ai[q] = fmaf(v.x, c.y, fmaf(v.y, c.x, ai[q]));
                }
            }
    }
    const float sg = ((k >> 1) & 1) ? -1.0f : 1.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = i0 + r + 4 * q;
        if (i < n_ant_pad) {
            const float hr = sg * ar[q], hi = sg * ai[q];
            grow[(size_t)i * CH_ROW + CH_HEADS + k] = make_float4(hr, hr, hi, hi);
        }
    }
}

struct ChebPointsArgs {
    const PtRec* pts;
    const float* vox;
    int64_t n;
    const float4* rows;        // [groups][n_ant_pad][CH_ROW]
    size_t group_rows;         // float4 per group of rows
    int ctas_per_group;        // point CTAs (blockIdx.x) per group
    int at;                    // antennas per tile
    int n_ant_tiles;
    int tiles_per_split;
    const ChebPlan* plan;
    const SplitPlan* gplan;    // per part (group, antenna block): interval and order
    int n_ab;                  // antenna blocks of CH_THREADS records with their own plan (1: one per group)
    const int* kmax;           // largest part order
    double k0;                 // K0 = 2 f_c / c at the band centre f_c, cycles per metre (positions in cycles)
    float gscale;              // gamma's 1 / (16 pi^2) per square cycle (render adjoint)
    float* partial;
    int* err;
};

// thread = 2 points (the two lanes of the packed Chebyshev sums)
static_assert(TPK_V == 2, "the packed Chebyshev sums carry two points per thread");

// A thread's two points, each quantity packed as (point 0, point 1): split
// position in cycles (h, l), and for the render adjoint the scaled normal
// n' = sqrt2 n, the transmittance T' and the directional offset, negated (-e).
struct PtPair {
    f2 hx, hy, hz, lx, ly, lz;
    f2 nx, ny, nz, te, ne;
};

__device__ __forceinline__ f2 dup2(float v) { return pk2(v, v); }

// One tile of AT antenna rows against this thread's two points, both points in
// the two lanes of every packed (f32x2) operation: the pair ranges in
// double-single (the split-coordinate form of pair_range_split, lane-wise),
// sum_k h_k T_k(x) for k < KE (KE even, fixed at compile time; rows are zero
// beyond the group's order), the carrier phasor, and the filter or
// render-adjoint accumulation into in. Only the square roots, the sincos and
// the rounding, clamps and masks run per lane. kGuard (the 64-order
// instance): orders past 32 run in blocks of 8 up to the group's own order K.
template <int MODE, int KE, bool kGuard>
__device__ __forceinline__ void points_tile(const float4* __restrict__ tile, int AT, int K, f2 INV, f2 HINV,
                                            const PtPair& P, f2 (&in)[MODE == MODE_FILTER ? 2 : 5]) {
    constexpr int ROW = CH_ROW;
    const f2 TWO = dup2(2.0f), NEG1 = dup2(-1.0f), HALF = dup2(0.5f);
#pragma unroll kPtsUnroll
    for (int a = 0; a < AT; ++a) {
        const ulonglong2* row = reinterpret_cast<const ulonglong2*>(tile + a * ROW);
        const ulonglong2 h0 = row[0], h1 = row[1], h2 = row[2], h3 = row[3];
        // h0 = (xh | yh), h1 = (zh | c_ant), h2 = (xl | yl), h3 = (zl | r_c), each in both lanes
        const f2 hx = sub2(P.hx, h0.x), hy = sub2(P.hy, h0.y), hz = sub2(P.hz, h1.x);
        const f2 lx = sub2(P.lx, h2.x), ly = sub2(P.ly, h2.y), lz = sub2(P.lz, h3.x);
        const f2 Sh = fma2(hz, hz, fma2(hy, hy, mul2(hx, hx)));              // exact
        const f2 cross = fma2(lx, fma2(TWO, hx, lx), fma2(ly, fma2(TWO, hy, ly), mul2(lz, fma2(TWO, hz, lz))));
        float s0, s1;
        upk2(add2(Sh, cross), s0, s1);
        s0 = fmaxf(s0, 1e-30f);
        s1 = fmaxf(s1, 1e-30f);
        const f2 S = pk2(s0, s1), RS = pk2(rsqrtf(s0), rsqrtf(s1));
        const f2 r0 = mul2(S, RS);                                           // range, leading part
        const f2 resid = add2(fma2(r0, mul2(r0, NEG1), Sh), cross);
        const f2 rl2 = mul2(resid, RS);                                      // one Newton step: r = r0 + rl2 / 2
        const f2 xs = fma2(rl2, HINV, mul2(sub2(r0, h3.y), INV));             // (r - r_c) / dr
        // sum_k h_k T_k(x) = sum_k (s_k h_k) V_k(x): V_k = s_k T_k for both
        // points in the two lanes of one packed FMA (V_k = (+/-2x) V_{k-1}
        // + V_{k-2}, minus for even k), the products accumulated for both
        // points at once; the rows carry s_k h_k and are zero beyond K,
        // so the loop may run to the next even order
        const ulonglong2* hk = row + CH_HEADS;
        const ulonglong2 h0u = hk[0], h1u = hk[1];
        const f2 mp = mul2(TWO, xs), mn = mul2(dup2(-2.0f), xs);
        f2 v0 = dup2(1.0f), v1 = xs;
        f2 Sr = h0u.x, Si = h0u.y;                       // V_0 = 1
        Sr = fma2(v1, h1u.x, Sr);
        Si = fma2(v1, h1u.y, Si);
#pragma unroll
        for (int kc = 0; kc < KE; kc += 8) {
            if (!kGuard || kc < 32 || kc < K) {
#pragma unroll
                for (int k = (kc == 0 ? 2 : kc); k < kc + 8 && k < KE; k += 2) {
                    const f2 ve = fma2(mn, v1, v0);
                    const ulonglong2 he = hk[k];
                    Sr = fma2(ve, he.x, Sr);
                    Si = fma2(ve, he.y, Si);
                    const f2 vo = fma2(mp, ve, v1);
                    const ulonglong2 ho = hk[k + 1];
                    Sr = fma2(vo, ho.x, Sr);
                    Si = fma2(vo, ho.y, Si);
                    v0 = ve;
                    v1 = vo;
                }
            }
        }
        // carrier phase in cycles: the fractional part of r0 + rl
        float a0, a1;
        upk2(r0, a0, a1);
        const f2 fr = fma2(rl2, HALF, sub2(r0, pk2(rintf(a0), rintf(a1))));
        float f0, f1;
        upk2(mul2(fr, dup2(6.28318530717958648f)), f0, f1);
        float sn0, cs0, sn1, cs1;
        __sincosf(f0, &sn0, &cs0);
        __sincosf(f1, &sn1, &cs1);
        const f2 CS = pk2(cs0, cs1), SN = pk2(sn0, sn1);
        if (MODE == MODE_FILTER) {
            // exp(+j 2 pi K0 r) * sum
            in[0] = fma2(CS, Sr, in[0]);
            in[0] = fma2(mul2(SN, NEG1), Si, in[0]);
            in[1] = fma2(CS, Si, in[1]);
            in[1] = fma2(SN, Sr, in[1]);
        } else {
            // q = Re(exp(-j 2 pi K0 r) * sum_k T_k H_k); with A = w T'^2 gamma D,
            // gamma = k16 / r^2 and n' = sqrt2 n: the sums below times the
            // per-point factors (k16, 2 w k16, 2 sqrt2 w k16, sqrt2 w k16) are
            // dA/dw, dA/dT', and the parts of dA/dn' along d and along n'
            const f2 q = fma2(SN, Si, mul2(CS, Sr));
            const f2 dx = add2(hx, lx), dy = add2(hy, ly), dz = add2(hz, lz);
            const f2 inv_r2 = mul2(RS, RS);
            const f2 g = mul2(q, inv_r2);
            const f2 nd = fma2(P.nz, dz, fma2(P.ny, dy, mul2(P.nx, dx)));
            const f2 Dm2 = fma2(mul2(nd, nd), inv_r2, P.ne);
            const f2 vv = sub2(P.te, h1.y);
            float dm0, dm1, vv0, vv1, ne0, ne1;
            upk2(Dm2, dm0, dm1);
            upk2(vv, vv0, vv1);
            upk2(P.ne, ne0, ne1);
            const float tt0 = __saturatef(vv0), tt1 = __saturatef(vv1);
            const f2 D = pk2(fmaxf(dm0, 0.0f), fmaxf(dm1, 0.0f));
            const f2 tg = mul2(pk2(tt0, tt1), g);
            const f2 u = mul2(pk2(tt0, tt1), tg);                            // T'^2 g
            in[0] = fma2(u, D, in[0]);
            // slope region 0 <= t_eff - c_ant <= 1 only (a per-lane select)
            float tg0, tg1;
            upk2(tg, tg0, tg1);
            in[1] = fma2(pk2(tt0 == vv0 ? tg0 : 0.0f, tt1 == vv1 ? tg1 : 0.0f), D, in[1]);
            // the directional factor's slope: e > 0 and D > 0 only
            float w0, w1;
            upk2(mul2(mul2(u, nd), inv_r2), w0, w1);
            const f2 w2 = pk2((ne0 < 0.0f && dm0 > 0.0f) ? w0 : 0.0f, (ne1 < 0.0f && dm1 > 0.0f) ? w1 : 0.0f);
            in[2] = fma2(w2, dx, in[2]);
            in[3] = fma2(w2, dy, in[3]);
            in[4] = fma2(w2, dz, in[4]);
        }
    }
}

#define GERAF_POINTS_CASE(E) \
    case E: points_tile<MODE, ((E) < KM ? (E) : KM), false>(tile, AT, K, INV, HINV, P, in); break;

// Each group of ctas_per_group point CTAs has its own interval and order
// (gplan) and its own antenna rows. KC = 8-order groups compiled in: the KC = 3
// and KC = 4 instances run when the largest group order is <= 24 or <= 32, each
// CTA with its part's order rounded up to even (at least 8) as a compile-time
// loop bound (one unrolled tile body per even order); the KC = 8 instance runs
// otherwise (orders beyond 32 guarded by the group's own order); all three are
// launched and the two that do not match return at once.
// Render adjoint: the per-point factors of the chain rule (the weight w, the
// constant 1/(16 pi^2) of gamma, and the numeric factors of dD/dn) are taken out
// of the antenna sums and applied once when the partials are written.
template <int MODE, int KC>
__global__ void __launch_bounds__(TPK_THREADS, KC <= 4 ? (MODE == MODE_FILTER ? GERAF_CH_FILTER_CTAS : GERAF_CH_RBWD_CTAS) : 1)
    cheb_points_kernel(const ChebPointsArgs args) {
    constexpr int KM = 8 * KC;
    if (!args.plan->run_cheb) return;
    {
        const int km = *args.kmax;
        if (KC != (km <= 24 ? 3 : (km <= 32 ? 4 : 8))) return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t* bar = reinterpret_cast<uint64_t*>(smem);
    int* abort_flag = reinterpret_cast<int*>(smem + 16);
    constexpr int ROW = CH_ROW;
    float4* rows = reinterpret_cast<float4*>(smem + 32);   // [2][at][ROW]
    const int AT = args.at;
    const int t = threadIdx.x;
    const int split = blockIdx.y;
    const int tile0 = split * args.tiles_per_split;
    const int tile1 = min(tile0 + args.tiles_per_split, args.n_ant_tiles);
    const int n_my = tile1 - tile0;
    const uint32_t tile_bytes = (uint32_t)(AT * ROW * sizeof(float4));
    const int grp = blockIdx.x / args.ctas_per_group;
    const float4* grows = args.rows + (size_t)grp * args.group_rows;
    if (t == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    if (t == 0)
        for (int s = 0; s < 2 && s < n_my; ++s) {
            mbar_arrive_expect_tx(&bar[s], tile_bytes);
            tma_load_1d(rows + s * AT * ROW, grows + (size_t)(tile0 + s) * AT * ROW, tile_bytes, &bar[s]);
        }
    const int64_t jbase = (blockIdx.x * (int64_t)TPK_THREADS + t) * TPK_V;
    float4 ph[TPK_V], pl[TPK_V];                             // split positions
    float pw[TPK_V], pnx[TPK_V], pny[TPK_V], pnz[TPK_V], pte[TPK_V], pe[TPK_V];
#pragma unroll
    for (int v = 0; v < TPK_V; ++v) {
        const int64_t j = min(jbase + v, args.n - 1);
        if (MODE == MODE_FILTER) {
            split3c(args.vox[j], args.vox[args.n + j], args.vox[2 * args.n + j], args.k0, ph[v], pl[v]);
            pw[v] = pnx[v] = pny[v] = pnz[v] = pte[v] = pe[v] = 0.0f;
        } else {
            const PtRec Q = args.pts[j];
            ph[v] = Q.a;
            pl[v] = Q.c;
            pw[v] = Q.a.w;
            pnx[v] = Q.b.x; pny[v] = Q.b.y; pnz[v] = Q.b.z; pte[v] = Q.b.w;
            pe[v] = Q.c.w;
        }
    }
    PtPair P;
    P.hx = pk2(ph[0].x, ph[1].x); P.hy = pk2(ph[0].y, ph[1].y); P.hz = pk2(ph[0].z, ph[1].z);
    P.lx = pk2(pl[0].x, pl[1].x); P.ly = pk2(pl[0].y, pl[1].y); P.lz = pk2(pl[0].z, pl[1].z);
    P.nx = pk2(pnx[0], pnx[1]); P.ny = pk2(pny[0], pny[1]); P.nz = pk2(pnz[0], pnz[1]);
    P.te = pk2(pte[0], pte[1]); P.ne = pk2(-pe[0], -pe[1]);
    // render adjoint: five sums; the sixth output, sum of w2 (n'.d), is n' dotted
    // with the three sums of w2 d and is formed at the end
    constexpr int NACC = (MODE == MODE_FILTER) ? 2 : 5;
    f2 hi[NACC], lo[NACC];                                   // Kahan sums over the tiles, both points
#pragma unroll
    for (int k = 0; k < NACC; ++k) hi[k] = lo[k] = pk2(0.0f, 0.0f);

    for (int it = 0; it < n_my; ++it) {
        const int buf = it & 1;
        if (!mbar_wait(&bar[buf], (it >> 1) & 1)) atomicOr(abort_flag, 1);
        __syncthreads();
        if (*abort_flag) {
            if (t == 0) {
                atomicOr(args.err, 1);
                mbar_drain2(bar, it, n_my);
            }
            return;
        }
        const float4* tile = rows + buf * AT * ROW;
        // the tile's part: its antenna block (AT divides CH_THREADS) of this group
        const SplitPlan gp =
            args.gplan[grp * args.n_ab + (args.n_ab > 1 ? ((tile0 + it) * AT) / CH_THREADS : 0)];
        const int K = gp.K;
        const int ke = K <= 8 ? 8 : (K + 1) & ~1;                // orders run: K rounded up to even, >= 8
        const f2 INV = dup2(gp.inv_dr), HINV = dup2(0.5f * gp.inv_dr);
        f2 in[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) in[k] = pk2(0.0f, 0.0f);
        if constexpr (KC == 8) {
            points_tile<MODE, KM, true>(tile, AT, K, INV, HINV, P, in);
        } else {
            switch (ke) {
                GERAF_POINTS_CASE(8) GERAF_POINTS_CASE(10) GERAF_POINTS_CASE(12) GERAF_POINTS_CASE(14)
                GERAF_POINTS_CASE(16) GERAF_POINTS_CASE(18) GERAF_POINTS_CASE(20) GERAF_POINTS_CASE(22)
                GERAF_POINTS_CASE(24) GERAF_POINTS_CASE(26) GERAF_POINTS_CASE(28) GERAF_POINTS_CASE(30)
                default: points_tile<MODE, KM, false>(tile, AT, K, INV, HINV, P, in);
            }
        }
#pragma unroll
        for (int k = 0; k < NACC; ++k) {
            const f2 y = sub2(in[k], lo[k]);
            const f2 sum = add2(hi[k], y);
            lo[k] = sub2(sub2(sum, hi[k]), y);
            hi[k] = sum;
        }
        __syncthreads();
        if (t == 0 && it + 2 < n_my) {
            mbar_arrive_expect_tx(&bar[buf], tile_bytes);
            tma_load_1d(rows + buf * AT * ROW, grows + (size_t)(tile0 + it + 2) * AT * ROW, tile_bytes,
                        &bar[buf]);
        }
    }
#pragma unroll
    for (int v = 0; v < TPK_V; ++v) {
        const int64_t j = jbase + v;
        if (j >= args.n) continue;
        float acc[NACC];
#pragma unroll
        for (int k = 0; k < NACC; ++k) {
            float h0, h1, l0, l1;
            upk2(hi[k], h0, h1);
            upk2(lo[k], l0, l1);
            acc[k] = v == 0 ? __fsub_rn(h0, l0) : __fsub_rn(h1, l1);
        }
        if (MODE == MODE_FILTER) {
            float2* dst = reinterpret_cast<float2*>(args.partial) + (size_t)split * args.n + j;
            *dst = make_float2(acc[0], acc[1]);
        } else {
            float* dst = args.partial + (size_t)split * 6 * args.n + j;
            const float wk = pw[v] * args.gscale;
            const float fac[6] = {args.gscale, 2.0f * wk, 2.0f * kSqrt2 * wk, 2.0f * kSqrt2 * wk, 2.0f * kSqrt2 * wk,
                                  kSqrt2 * wk};
            float sum[6];
#pragma unroll
            for (int k = 0; k < 5; ++k) sum[k] = acc[k];
            sum[5] = pnx[v] * sum[2] + pny[v] * sum[3] + pnz[v] * sum[4];
#pragma unroll
            for (int k = 0; k < 6; ++k) dst[(size_t)k * args.n] = sum[k] * fac[k];
        }
    }
}

bool use_cheb(const geraf_band* band) {
    if (band->method == GERAF_PHASOR_RECURRENCE) return false;
    if (band->method == GERAF_PHASOR_CHEBYSHEV) return true;
    return band->n_f >= 64;
}

// K0 = 2 f_c / c with f_c = f0 + (n_f - 1) df / 2 the band's centre: carrier
// cycles per metre of range (the Chebyshev kernels' coordinate unit)
double k0_of(const geraf_band* band) { return 2.0 * (band->f0 + 0.5 * (band->n_f - 1) * band->df) / kC; }

// Kc = df / f_c: the bin phase step in cycles per cycle of range
double kc_of(const geraf_band* band) { return band->df / (band->f0 + 0.5 * (band->n_f - 1) * band->df); }

// 1 / (16 pi^2) per square cycle of range, the factor of gamma = 1 / (4 pi r)^2
// for ranges in cycles
float gamma_scale(const geraf_band* band) {
    const double k0 = k0_of(band);
    return (float)(0.0063325739776461107 * k0 * k0);
}

geraf_status check_launch(const char* what) { return cuda_status(cudaGetLastError(), what); }

inline unsigned grid1d(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

// ============================================================== entry points

namespace {

struct ChebWs {
    float* bbox;
    ChebPlan* plan;
    int n_bbox_blocks;
};

ChebWs take_cheb(WsCarver& c, int64_t n_bbox) {
    ChebWs w;
    w.n_bbox_blocks = (int)std::min<int64_t>((n_bbox + 255) / 256, 1024);
    w.bbox = c.take<float>((size_t)w.n_bbox_blocks * 6);
    w.plan = c.take<ChebPlan>(1);
    return w;
}

// Point groups of the to-points calls: consecutive point CTAs, each group with
// its own antenna rows (at most GERAF_CH_MAX_GROUPS groups and CH_GROUP_ROWS_BYTES of rows; at
// least 8 CTAs = 2048 points per group), planned per (group, block of
// CH_THREADS antenna records in the spatial order) while the parts' tables fit
// CH_TABLE_BYTES, else per group over all antennas.
constexpr size_t CH_GROUP_ROWS_BYTES = (size_t)GERAF_CH_GROUP_ROWS_MIB << 20;
struct PointGroups {
    int groups, ctas_per_group, n_ab, parts;
    float* box;
    SplitPlan* plan;
    float* rcs;          // [groups][n_ant_pad]: each antenna record's range centre per group
    float2* C;
    int* kmax;
    float4* rows;
    size_t group_rows;
};
PointGroups plan_point_groups(int pt_ctas, int n_ant, int n_ant_pad, int n_f) {
    PointGroups g{};
    g.group_rows = (size_t)n_ant_pad * CH_ROW;
    const size_t cap = std::max<size_t>(
        1, std::min<size_t>(GERAF_CH_MAX_GROUPS, CH_GROUP_ROWS_BYTES / (g.group_rows * sizeof(float4))));
    g.ctas_per_group = std::max<int>(8, (int)((pt_ctas + cap - 1) / cap));
    g.groups = (pt_ctas + g.ctas_per_group - 1) / g.ctas_per_group;
    const int nb = (n_ant + CH_THREADS - 1) / CH_THREADS;
    const size_t table = (size_t)CH_KMAX * n_f * sizeof(float2);
    g.n_ab = (nb > 1 && (size_t)g.groups * nb * table <= CH_TABLE_BYTES) ? nb : 1;
    g.parts = g.groups * g.n_ab;
    return g;
}
PointGroups take_point_groups(WsCarver& c, int pt_ctas, int n_ant, int n_ant_pad, int n_f) {
    PointGroups g = plan_point_groups(pt_ctas, n_ant, n_ant_pad, n_f);
    g.box = c.take<float>((size_t)g.groups * 6);
    g.plan = c.take<SplitPlan>(g.parts);
    g.rcs = c.take<float>((size_t)g.groups * n_ant_pad);
    g.C = c.take<float2>((size_t)g.parts * CH_KMAX * n_f);
    g.kmax = c.take<int>(1);
    g.rows = c.take<float4>((size_t)g.groups * g.group_rows);
    return g;
}

// Spatial order of the antennas and their records in it (Chebyshev calls)
struct AntOrder {
    int* perm;
    float4* rec;
    unsigned long long* sort_buf;   // the sort's global scratch when it does not fit in shared memory
    int n_rec, n_pow2;
};
AntOrder take_ant_order(WsCarver& c, int n_ant, int n_rec) {
    AntOrder a{};
    a.n_rec = n_rec;
    a.n_pow2 = pow2_at_least(n_ant);
    a.perm = c.take<int>(n_rec);
    a.rec = c.take<float4>(n_rec);
    a.sort_buf = a.n_pow2 > AO_SMEM_MAX ? c.take<unsigned long long>(a.n_pow2) : nullptr;
    return a;
}
void launch_ant_order(const AntOrder& a, const float* ant_xyz, const float* c_ant, int n_ant, cudaStream_t st) {
    antenna_order_kernel<<<1, AO_THREADS, antenna_order_smem(a.n_pow2), st>>>(ant_xyz, n_ant, a.n_pow2, a.sort_buf,
                                                                              a.perm, a.n_rec);
    pack_antennas_perm<<<grid1d(a.n_rec, 256), 256, 0, st>>>(ant_xyz, c_ant, n_ant, a.perm, a.n_rec, a.rec);
}

// Brick order of the points (Chebyshev calls): perm and the sort's buffers
struct PointOrder {
    int* perm;
    uint16_t* bkt;
    int* hist;
    int* seg;
    int* base;
    int64_t n, n_sub;
    int n_seg;
    unsigned blocks;
};
PointOrder take_point_order(WsCarver& c, int64_t n) {
    PointOrder o{};
    o.n = n;
    o.blocks = (unsigned)((n + (int64_t)PO_SUB * PO_WARPS - 1) / ((int64_t)PO_SUB * PO_WARPS));
    o.n_sub = (int64_t)o.blocks * PO_WARPS;          // every warp's sub-chunk, empty ones included
    o.n_seg = (int)((o.n_sub + PO_SEG - 1) / PO_SEG);
    o.perm = c.take<int>((size_t)n);
    o.bkt = c.take<uint16_t>((size_t)n);
    o.hist = c.take<int>((size_t)o.n_sub * PO_BUCKETS);
    o.seg = c.take<int>((size_t)o.n_seg * PO_BUCKETS);
    o.base = c.take<int>(PO_BUCKETS);
    return o;
}
void launch_point_order(const PointOrder& o, const float* xyz, const ChebPlan* plan, cudaStream_t st) {
    point_hist_kernel<<<o.blocks, 32 * PO_WARPS, 0, st>>>(xyz, o.n, plan, o.bkt, o.hist);
    point_scan_segments<<<o.n_seg, PO_BUCKETS, 0, st>>>(o.hist, o.n_sub, o.seg);
    point_scan_totals<<<1, PO_BUCKETS, 0, st>>>(o.seg, o.n_seg, o.base);
    point_scatter_kernel<<<o.blocks, 32 * PO_WARPS, 0, st>>>(o.bkt, o.n, o.hist, o.seg, o.base, o.perm);
}

// group boxes, part plans and tables, then the groups' antenna rows
geraf_status launch_point_groups(const PointGroups& g, const ChebWs& cw, const AntOrder& ao, const float* xyz,
                                 int64_t n, const float* ant_xyz, const float* c_ant, int n_ant, int n_ant_pad,
                                 const geraf_band* band, const float2* sig, int conj_c, int conj_sig,
                                 cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(g.kmax, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e, "point groups");
    group_bbox_kernel<<<g.groups, 256, 0, st>>>(xyz, n, (int64_t)g.ctas_per_group * TPK_THREADS * TPK_V,
                                                (float)k0_of(band), g.box);
    split_plan_kernel<<<g.parts, 256, 0, st>>>(g.box, ao.rec, n_ant, n_ant_pad, g.n_ab,
                                               g.n_ab > 1 ? CH_THREADS : n_ant, 2.0 * band->df / kC, band->n_f,
                                               CH_TAIL, k0_of(band), cw.plan, g.plan, g.rcs, g.C, g.kmax);
    cheb_group_rows_kernel<<<dim3((n_ant_pad + GR_T - 1) / GR_T, g.groups), 256, 0, st>>>(
        ant_xyz, c_ant, sig, ao.perm, n_ant, n_ant_pad, band->n_f, g.n_ab, cw.plan, g.plan, g.C, g.rcs,
        kc_of(band), conj_c, conj_sig, k0_of(band), g.rows);
    return GERAF_OK;
}

void launch_cheb_plan(const ChebWs& w, const float* pts, int64_t n, const float* ant, int n_ant,
                      const geraf_band* band, cudaStream_t st) {
    bbox_partial_kernel<<<w.n_bbox_blocks, 256, 0, st>>>(pts, n, w.bbox);
    cheb_plan_kernel<<<1, 256, 0, st>>>(w.bbox, w.n_bbox_blocks, ant, n_ant, 2.0 * band->df / kC, band->n_f, CH_TAIL,
                                        k0_of(band), w.plan);
}

struct ChebBinsPlan {
    int ant_blocks, n_tiles, splits, tiles_per_split;
    int plan_blocks;     // antenna blocks with their own plan per split (1: one plan per split)
};

ChebBinsPlan plan_cheb_bins(int64_t n_pad, int n_ant, int n_f) {
    ChebBinsPlan q;
    q.ant_blocks = (n_ant + CH_THREADS - 1) / CH_THREADS;
    q.n_tiles = (int)(n_pad / CH_TP);
    const int64_t max_splits = std::max<int64_t>(1, (int64_t)(CH_PARTIAL_BYTES / ((size_t)n_ant * CH_KMAX * 8)));
    int64_t want = std::max<int64_t>(
        1, ((int64_t)GERAF_CH_SPLIT_CTAS_PER_SM * device_sm_count() + q.ant_blocks - 1) / q.ant_blocks);
    // as many splits of at least GERAF_CH_SPLIT_MIN_PTS points as there is
    // room for: each split is then a compact brick of the point order, and
    // splits of that size get a plan per antenna block
    want = std::max<int64_t>(want, n_pad / GERAF_CH_SPLIT_MIN_PTS);
    // at most GERAF_CH_MAX_SPLITS splits; each part (a split, or a split and an
    // antenna block) carries its own coefficient table
    const int64_t sp = std::min<int64_t>(std::min<int64_t>(std::min<int64_t>(max_splits, want), q.n_tiles),
                                         GERAF_CH_MAX_SPLITS);
    q.tiles_per_split = (int)((q.n_tiles + sp - 1) / sp);
    q.splits = (q.n_tiles + q.tiles_per_split - 1) / q.tiles_per_split;
    // a plan per (split, antenna block) pays when a part holds enough pairs to
    // outweigh its plan (Bessel values of every bin): splits of at least
    // 8192 points, and at most CH_TABLE_BYTES of tables; otherwise one plan per split
    const int64_t max_parts = std::max<int64_t>(1, (int64_t)(CH_TABLE_BYTES / ((size_t)CH_KMAX * n_f * 8)));
    const bool blocks = (int64_t)q.tiles_per_split * CH_TP >= GERAF_CH_SPLIT_MIN_PTS && (int64_t)q.splits * q.ant_blocks <= max_parts;
    q.plan_blocks = blocks ? q.ant_blocks : 1;
    return q;
}

template <bool kComplexAmp>
geraf_status to_bins_call(int64_t n_pts, const float* ant_xyz, const float* c_ant, int32_t n_ant,
                          const geraf_band* band, int32_t flags, const float* xyz, const float* grad, const float* w,
                          const float* t_eff, const float* vox, const float2* M, const float* dP, void* ws,
                          size_t* ws_bytes, float* out, cudaStream_t st, const char* name) {
    // render packs points xyz (weights w, t_eff, grad); the filter adjoint packs voxels vox (M, dP)
    const float* positions = kComplexAmp ? vox : xyz;
    BandK bk;
    if (!make_band_k(band, &bk)) return GERAF_ERR_INVALID_ARG;
    const bool cheb = use_cheb(band);
    const int64_t n_pad = cheb ? (n_pts + CH_TP - 1) / CH_TP * CH_TP : n_pts;
    ToBinsPlan p = plan_to_bins(n_pad, n_ant, bk.g);
    const int64_t n_rec = (int64_t)p.n_tiles * p.TP;
    const int n_ant_rec = std::max(p.n_ant_pad, (n_ant + CH_THREADS - 1) / CH_THREADS * CH_THREADS);
    ChebBinsPlan q{};
    if (cheb) q = plan_cheb_bins(n_rec, n_ant, band->n_f);
    const int parts = q.splits * q.plan_blocks;
    WsCarver c(ws);
    PtRec* pts = c.take<PtRec>((size_t)n_rec);
    float4* ant = c.take<float4>(n_ant_rec);
    float2* part = c.take<float2>((size_t)p.splits * p.n_ant_pad * 32 * p.G);
    ChebWs cw{};
    AntOrder ao{};
    float2* cpart = nullptr;
    float* sbox = nullptr;
    SplitPlan* splan = nullptr;
    float* srcs = nullptr;
    float2* scs = nullptr;
    int* kmax = nullptr;
    float2* gout = nullptr;
    PointOrder po{};
    if (cheb) {
        cw = take_cheb(c, n_pts);
        ao = take_ant_order(c, n_ant, n_ant_rec);
        po = take_point_order(c, n_pts);
        cpart = c.take<float2>((size_t)q.splits * n_ant * CH_KMAX);
        sbox = c.take<float>((size_t)q.splits * 6);
        splan = c.take<SplitPlan>(parts);
        srcs = c.take<float>((size_t)q.splits * n_ant_rec);
        scs = c.take<float2>((size_t)parts * CH_KMAX * band->n_f);
        kmax = c.take<int>(1);
        gout = c.take<float2>((size_t)((q.splits + RS - 1) / RS) * n_ant * band->n_f);
    }
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used) return fail(GERAF_ERR_WORKSPACE, "%s: workspace %zu < %zu bytes", name, *ws_bytes, c.used);
    int* err = device_error_word();
    {
        const geraf_status as = smem_attrs(200 * 1024, "shared-memory opt-in", to_bins_kernel<false>,
                                           to_bins_kernel<true>, cheb_bins_kernel<false, 3>,
                                           cheb_bins_kernel<true, 3>, cheb_bins_kernel<false, 4>,
                                           cheb_bins_kernel<true, 4>, cheb_bins_kernel<false, 8>,
                                           cheb_bins_kernel<true, 8>, antenna_order_kernel);
        if (as != GERAF_OK) return as;
    }
    if (cheb) {
        // whole-call plan (and the points' box), then the points in brick order
        launch_cheb_plan(cw, positions, n_pts, ant_xyz, n_ant, band, st);
        launch_point_order(po, positions, cw.plan, st);
    }
    if (!kComplexAmp)
        pack_render_points<<<grid1d(n_rec, 256), 256, 0, st>>>(xyz, grad, w, t_eff, n_pts, n_rec,
                                                               (flags & GERAF_RENDER_DIRECTIONAL) ? 1 : 0, pts,
                                                               po.perm, cheb ? &cw.plan->run_cheb : nullptr,
                                                               k0_of(band), 1);
    else
        pack_filter_bwd_points<<<grid1d(n_rec, 256), 256, 0, st>>>(vox, M, dP, n_pts, n_rec, pts, po.perm,
                                                                   cheb ? &cw.plan->run_cheb : nullptr,
                                                                   k0_of(band), 1);
    pack_antennas<<<grid1d(n_ant_rec, 256), 256, 0, st>>>(ant_xyz, c_ant, n_ant, n_ant_rec, ant);
    const int* run_direct = nullptr;
    if (cheb) {
        launch_ant_order(ao, ant_xyz, c_ant, n_ant, st);
        cudaError_t e = cudaMemsetAsync(kmax, 0, sizeof(int), st);
        if (e != cudaSuccess) return cuda_status(e, name);
        split_bbox_kernel<<<q.splits, 256, 0, st>>>(pts, q.n_tiles, q.tiles_per_split, sbox);
        split_plan_kernel<<<parts, 256, 0, st>>>(sbox, ao.rec, n_ant, n_ant_rec, q.plan_blocks,
                                                 q.plan_blocks > 1 ? CH_THREADS : n_ant, 2.0 * band->df / kC,
                                                 band->n_f, CH_TAIL, k0_of(band), cw.plan, splan, srcs, scs, kmax);
        ChebBinsArgs ca{pts,    ao.rec, n_ant, q.n_tiles, q.tiles_per_split,   cw.plan,
                        splan,  q.plan_blocks, srcs, n_ant_rec, kmax, k0_of(band),
                        kComplexAmp ? 1.0f : gamma_scale(band), cpart,  err};
        const dim3 grid(q.ant_blocks, q.splits);
        cheb_bins_kernel<kComplexAmp, 3><<<grid, CH_THREADS, cheb_bins_smem(24), st>>>(ca);
        cheb_bins_kernel<kComplexAmp, 4><<<grid, CH_THREADS, cheb_bins_smem(32), st>>>(ca);
        cheb_bins_kernel<kComplexAmp, 8><<<grid, CH_THREADS, cheb_bins_smem(64), st>>>(ca);
        const int groups = (q.splits + RS - 1) / RS;
        cheb_reconstruct_split_kernel<<<dim3((n_ant + RA - 1) / RA, groups), 128, 0, st>>>(
            cpart, q.splits, n_ant, band->n_f, q.plan_blocks, cw.plan, splan, scs, srcs, n_ant_rec, kc_of(band),
            ao.perm, gout);
        sum_split_groups<<<grid1d((int64_t)n_ant * band->n_f, 256), 256, 0, st>>>(
            gout, groups, (int64_t)n_ant * band->n_f, cw.plan, reinterpret_cast<float2*>(out));
        run_direct = &cw.plan->use_direct;
    }
    ToBinsArgs a{pts, ant, part, err, p.TP, p.n_tiles, p.tiles_per_split, p.n_ant_pad, p.A_T, bk, run_direct};
    to_bins_kernel<kComplexAmp><<<dim3(p.ant_ctas, p.splits), TB_THREADS, p.smem, st>>>(a);
    reduce_bins<<<grid1d((int64_t)n_ant * band->n_f, 256), 256, 0, st>>>(part, p.splits, n_ant, p.n_ant_pad,
                                                                         band->n_f, 32 * p.G,
                                                                         reinterpret_cast<float2*>(out), run_direct);
    return check_launch(name);
}

}  // namespace

geraf_status render_impl(const float* xyz, const float* grad, const float* w, const float* t_eff, int64_t n_pts,
                         const float* ant_xyz, const float* c_ant, int32_t n_ant, const geraf_band* band,
                         int32_t flags, void* ws, size_t* ws_bytes, float* s_out, cudaStream_t st) {
    return to_bins_call<false>(n_pts, ant_xyz, c_ant, n_ant, band, flags, xyz, grad, w, t_eff, nullptr, nullptr,
                               nullptr, ws, ws_bytes, s_out, st, "render");
}

geraf_status filter_backward_impl(const float* ant_xyz, int32_t n_ant, const geraf_band* band, const float* vox,
                                  int64_t n_vox, const float* M, const float* d_P, void* ws, size_t* ws_bytes,
                                  float* g_s, cudaStream_t st) {
    return to_bins_call<true>(n_vox, ant_xyz, nullptr, n_ant, band, 0, nullptr, nullptr, nullptr, nullptr, vox,
                              reinterpret_cast<const float2*>(M), d_P, ws, ws_bytes, g_s, st, "filter_backward");
}

geraf_status filter_impl(const float* s, const float* ant_xyz, int32_t n_ant, const geraf_band* band,
                         const float* vox, int64_t n_vox, const float* target, const float* mask, void* ws,
                         size_t* ws_bytes, float* P, float* M, double* loss, float* dloss_dP, cudaStream_t st) {
    BandK bk;
    if (!make_band_k(band, &bk)) return GERAF_ERR_INVALID_ARG;
    const bool cheb = use_cheb(band);
    ToPointsPlan p = plan_to_points(n_vox, n_ant, bk.g);
    const ChebPointsTiles cq = cheb_points_tiles(p, n_ant);
    WsCarver c(ws);
    float4* rows = c.take<float4>((size_t)p.n_ant_pad * p.row_f4);
    float2* part = c.take<float2>((size_t)p.splits * n_vox);
    const int fin_blocks = (int)grid1d(n_vox, 256);
    double* loss_blocks = c.take<double>(fin_blocks);
    ChebWs cw{};
    PointGroups pg{};
    AntOrder ao{};
    PointOrder po{};
    float* vox_p = nullptr;
    if (cheb) {
        cw = take_cheb(c, n_vox);
        pg = take_point_groups(c, p.pt_ctas, n_ant, cq.n_ant_pad, band->n_f);
        ao = take_ant_order(c, n_ant, cq.n_ant_pad);
        po = take_point_order(c, n_vox);
        vox_p = c.take<float>((size_t)3 * n_vox);
    }
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used) return fail(GERAF_ERR_WORKSPACE, "filter: workspace %zu < %zu bytes", *ws_bytes, c.used);
    int* err = device_error_word();
    {
        const geraf_status as = smem_attrs(200 * 1024, "shared-memory opt-in", to_points_kernel<MODE_FILTER>,
                                           cheb_points_kernel<MODE_FILTER, 3>, cheb_points_kernel<MODE_FILTER, 4>,
                                           cheb_points_kernel<MODE_FILTER, 8>, antenna_order_kernel);
        if (as != GERAF_OK) return as;
    }
    const int* run_direct = nullptr;
    if (cheb) {
        launch_cheb_plan(cw, vox, n_vox, ant_xyz, n_ant, band, st);
        launch_point_order(po, vox, cw.plan, st);
        gather_xyz<<<grid1d(n_vox, 256), 256, 0, st>>>(vox, n_vox, po.perm, vox_p);
        launch_ant_order(ao, ant_xyz, nullptr, n_ant, st);
        const geraf_status gs = launch_point_groups(pg, cw, ao, vox_p, n_vox, ant_xyz, nullptr, n_ant, cq.n_ant_pad,
                                                    band, reinterpret_cast<const float2*>(s), 1, 0, st);
        if (gs != GERAF_OK) return gs;
        ChebPointsArgs ca{nullptr, vox_p, n_vox, pg.rows, pg.group_rows, pg.ctas_per_group, cq.at, cq.n_ant_tiles,
                          cq.tiles_per_split, cw.plan, pg.plan, pg.n_ab, pg.kmax, k0_of(band), 1.0f,
                          reinterpret_cast<float*>(part), err};
        const size_t smem = 32 + 2 * (size_t)cq.at * CH_ROW * sizeof(float4);
        cheb_points_kernel<MODE_FILTER, 3><<<dim3(p.pt_ctas, p.splits), TPK_THREADS, smem, st>>>(ca);
        cheb_points_kernel<MODE_FILTER, 4><<<dim3(p.pt_ctas, p.splits), TPK_THREADS, smem, st>>>(ca);
        cheb_points_kernel<MODE_FILTER, 8><<<dim3(p.pt_ctas, p.splits), TPK_THREADS, smem, st>>>(ca);
        run_direct = &cw.plan->use_direct;
    }
    pack_antenna_rows<<<p.n_ant_pad, 128, 0, st>>>(ant_xyz, nullptr, reinterpret_cast<const float2*>(s), n_ant,
                                                   p.n_ant_pad, band->n_f, p.n_f_pad, rows, run_direct);
    ToPointsArgs a{nullptr, cheb ? vox_p : vox, n_vox, rows, p.row_f4, p.at, p.n_ant_tiles, p.tiles_per_split,
                   reinterpret_cast<float*>(part), err, bk, run_direct};
    to_points_kernel<MODE_FILTER><<<dim3(p.pt_ctas, p.splits), TPK_THREADS, p.smem, st>>>(a);
    const bool want_loss = target != nullptr;
    filter_finalize<<<fin_blocks, 256, 0, st>>>(part, p.splits, n_vox, target, mask, P,
                                                reinterpret_cast<float2*>(M), want_loss ? dloss_dP : nullptr,
                                                want_loss ? loss_blocks : nullptr, po.perm);
    if (want_loss && loss) sum_doubles<<<1, 256, 0, st>>>(loss_blocks, fin_blocks, loss);
    return check_launch("filter");
}

geraf_status render_backward_impl(const float* xyz, const float* grad, const float* w, const float* t_eff,
                                  int64_t n_pts, const float* ant_xyz, const float* c_ant, int32_t n_ant,
                                  const geraf_band* band, int32_t flags, const float* g_s, void* ws,
                                  size_t* ws_bytes, float* d_w, float* d_teff, float* d_grad, cudaStream_t st) {
    BandK bk;
    if (!make_band_k(band, &bk)) return GERAF_ERR_INVALID_ARG;
    const bool cheb = use_cheb(band);
    ToPointsPlan p = plan_to_points(n_pts, n_ant, bk.g);
    const ChebPointsTiles cq = cheb_points_tiles(p, n_ant);
    WsCarver c(ws);
    PtRec* pts = c.take<PtRec>((size_t)n_pts);
    float4* rows = c.take<float4>((size_t)p.n_ant_pad * p.row_f4);
    float* part = c.take<float>((size_t)p.splits * 6 * n_pts);
    ChebWs cw{};
    PointGroups pg{};
    AntOrder ao{};
    PointOrder po{};
    float* xyz_p = nullptr;
    if (cheb) {
        cw = take_cheb(c, n_pts);
        pg = take_point_groups(c, p.pt_ctas, n_ant, cq.n_ant_pad, band->n_f);
        ao = take_ant_order(c, n_ant, cq.n_ant_pad);
        po = take_point_order(c, n_pts);
        xyz_p = c.take<float>((size_t)3 * n_pts);
    }
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used)
        return fail(GERAF_ERR_WORKSPACE, "render_backward: workspace %zu < %zu bytes", *ws_bytes, c.used);
    int* err = device_error_word();
    if (cheb) {
        // whole-call plan (and the points' box), then the points in brick order
        launch_cheb_plan(cw, xyz, n_pts, ant_xyz, n_ant, band, st);
        launch_point_order(po, xyz, cw.plan, st);
        gather_xyz<<<grid1d(n_pts, 256), 256, 0, st>>>(xyz, n_pts, po.perm, xyz_p);
    }
    pack_render_points<<<grid1d(n_pts, 256), 256, 0, st>>>(xyz, grad, w, t_eff, n_pts, n_pts,
                                                           (flags & GERAF_RENDER_DIRECTIONAL) ? 1 : 0, pts, po.perm,
                                                           cheb ? &cw.plan->run_cheb : nullptr, k0_of(band));
    {
        const geraf_status as = smem_attrs(200 * 1024, "shared-memory opt-in", to_points_kernel<MODE_RENDER_BWD>,
                                           cheb_points_kernel<MODE_RENDER_BWD, 3>,
                                           cheb_points_kernel<MODE_RENDER_BWD, 4>,
                                           cheb_points_kernel<MODE_RENDER_BWD, 8>, antenna_order_kernel);
        if (as != GERAF_OK) return as;
    }
    const int* run_direct = nullptr;
    if (cheb) {
        launch_ant_order(ao, ant_xyz, c_ant, n_ant, st);
        const geraf_status gs = launch_point_groups(pg, cw, ao, xyz_p, n_pts, ant_xyz, c_ant, n_ant, cq.n_ant_pad,
                                                    band, reinterpret_cast<const float2*>(g_s), 0, 1, st);
        if (gs != GERAF_OK) return gs;
        ChebPointsArgs ca{pts,     nullptr,  n_pts,      pg.rows,     pg.group_rows,       pg.ctas_per_group,
                          cq.at,   cq.n_ant_tiles, cq.tiles_per_split, cw.plan, pg.plan, pg.n_ab,
                          pg.kmax, k0_of(band),   gamma_scale(band), part,    err};
        const size_t smem = 32 + 2 * (size_t)cq.at * CH_ROW * sizeof(float4);
        cheb_points_kernel<MODE_RENDER_BWD, 3><<<dim3(p.pt_ctas, p.splits), TPK_THREADS, smem, st>>>(ca);
        cheb_points_kernel<MODE_RENDER_BWD, 4><<<dim3(p.pt_ctas, p.splits), TPK_THREADS, smem, st>>>(ca);
        cheb_points_kernel<MODE_RENDER_BWD, 8><<<dim3(p.pt_ctas, p.splits), TPK_THREADS, smem, st>>>(ca);
        run_direct = &cw.plan->use_direct;
    }
    pack_antenna_rows<<<p.n_ant_pad, 128, 0, st>>>(ant_xyz, c_ant, reinterpret_cast<const float2*>(g_s), n_ant,
                                                   p.n_ant_pad, band->n_f, p.n_f_pad, rows, run_direct);
    ToPointsArgs a{pts, nullptr, n_pts, rows, p.row_f4, p.at, p.n_ant_tiles, p.tiles_per_split, part, err, bk,
                   run_direct};
    to_points_kernel<MODE_RENDER_BWD><<<dim3(p.pt_ctas, p.splits), TPK_THREADS, p.smem, st>>>(a);
    render_bwd_finalize<<<grid1d(n_pts, 256), 256, 0, st>>>(part, p.splits, n_pts, pts, grad,
                                                            (flags & GERAF_RENDER_DIRECTIONAL) ? 1 : 0, d_w,
                                                            d_teff, d_grad, po.perm);
    return check_launch("render_backward");
}

namespace {
// dynamic loss mask, masked L2 loss (FP64 block partials), its gradient and
// the running maximum of P, one voxel per thread
__global__ void masked_loss_kernel(const float* __restrict__ P, const float* __restrict__ target,
                                   float* __restrict__ hist, int64_t n, float t_hi, float t_lo,
                                   float* __restrict__ mask, float* __restrict__ dP, double* __restrict__ blocks) {
    __shared__ double red[256];
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double l = 0.0;
    if (i < n) {
        const float p = P[i], h = hist[i];
        const float m = (h >= t_hi && p < t_lo) ? 0.0f : 1.0f;
        const float r = p - target[i];
        l = (double)m * (double)r * (double)r;
        if (dP) dP[i] = 2.0f * m * r;
        if (mask) mask[i] = m;
        hist[i] = fmaxf(h, p);
    }
    red[threadIdx.x] = l;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) blocks[blockIdx.x] = red[0];
}
}  // namespace

geraf_status masked_loss_impl(const float* P, const float* target, float* history, int64_t n_vox, float t_hi,
                              float t_lo, void* ws, size_t* ws_bytes, double* loss, float* dloss_dP, float* mask,
                              cudaStream_t st) {
    const int blocks = (int)grid1d(n_vox, 256);
    WsCarver c(ws);
    double* part = c.take<double>(blocks);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used) return fail(GERAF_ERR_WORKSPACE, "masked_loss: workspace %zu < %zu bytes", *ws_bytes, c.used);
    masked_loss_kernel<<<blocks, 256, 0, st>>>(P, target, history, n_vox, t_hi, t_lo, mask, dloss_dP, part);
    sum_doubles<<<1, 256, 0, st>>>(part, blocks, loss);
    return check_launch("masked_loss");
}

geraf_status chebyshev_order_impl(const float* xyz, int64_t n, const float* ant_xyz, int32_t n_ant,
                                  const geraf_band* band, void* ws, size_t* ws_bytes, int32_t* order,
                                  cudaStream_t st) {
    BandK bk;
    if (!make_band_k(band, &bk)) return GERAF_ERR_INVALID_ARG;
    WsCarver c(ws);
    ChebWs cw = take_cheb(c, n);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used)
        return fail(GERAF_ERR_WORKSPACE, "chebyshev_order: workspace %zu < %zu bytes", *ws_bytes, c.used);
    if (!use_cheb(band)) {
        *order = 0;
        return GERAF_OK;
    }
    launch_cheb_plan(cw, xyz, n, ant_xyz, n_ant, band, st);
    geraf_status s = check_launch("chebyshev_order");
    if (s != GERAF_OK) return s;
    ChebPlan h;
    cudaError_t e = cudaMemcpyAsync(&h, cw.plan, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "chebyshev_order: read back");
    *order = h.use_direct ? 0 : h.K;
    return GERAF_OK;
}

// Orders one Chebyshev phasor call evaluates: the same device plans as the
// call (whole set; the antennas in the spatial order; then per part = split of
// point tiles or point group, times a block of antenna records where the call
// plans per block), read back; the kernel instance follows the largest part
// order (24, 32 or 64 orders compiled in; the 64-order instance runs 32 orders
// plus the part's own beyond them, in blocks of 8; the others the part's order
// rounded up to even, at least 8). mean_orders = orders per (point, antenna)
// pair, averaged over all pairs.
geraf_status chebyshev_work_impl(const float* xyz, int64_t n, const float* ant_xyz, int32_t n_ant,
                                 const geraf_band* band, int32_t to_points, void* ws, size_t* ws_bytes,
                                 int32_t* orders, double* mean_orders, cudaStream_t st) {
    BandK bk;
    if (!make_band_k(band, &bk)) return GERAF_ERR_INVALID_ARG;
    int parts = 0, n_ab = 1, ant_per_block = n_ant, n_rec = 0;
    int64_t per_part = 0;
    if (to_points) {
        const ToPointsPlan p = plan_to_points(n, n_ant, bk.g);
        const PointGroups g = plan_point_groups(p.pt_ctas, n_ant, cheb_points_tiles(p, n_ant).n_ant_pad, band->n_f);
        n_ab = g.n_ab;
        parts = g.parts;
        per_part = (int64_t)g.ctas_per_group * TPK_THREADS * TPK_V;
        n_rec = cheb_points_tiles(p, n_ant).n_ant_pad;
    } else {
        const int64_t n_pad = (n + CH_TP - 1) / CH_TP * CH_TP;
        const ToBinsPlan p = plan_to_bins(n_pad, n_ant, bk.g);
        const ChebBinsPlan q = plan_cheb_bins((int64_t)p.n_tiles * p.TP, n_ant, band->n_f);
        n_ab = q.plan_blocks;
        parts = q.splits * n_ab;
        per_part = (int64_t)q.tiles_per_split * CH_TP;
        n_rec = std::max(p.n_ant_pad, (n_ant + CH_THREADS - 1) / CH_THREADS * CH_THREADS);
    }
    ant_per_block = n_ab > 1 ? CH_THREADS : n_ant;
    const int n_splits = parts / n_ab;
    WsCarver c(ws);
    ChebWs cw = take_cheb(c, n);
    AntOrder ao = take_ant_order(c, n_ant, n_rec);
    PointOrder po = take_point_order(c, n);
    float* xyz_p = c.take<float>((size_t)3 * n);
    float* box = c.take<float>((size_t)n_splits * 6);
    SplitPlan* splan = c.take<SplitPlan>(parts);
    float* rcs = c.take<float>((size_t)n_splits * n_rec);
    float2* Cs = c.take<float2>((size_t)parts * CH_KMAX * band->n_f);
    int* kmax = c.take<int>(1);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used)
        return fail(GERAF_ERR_WORKSPACE, "chebyshev_work: workspace %zu < %zu bytes", *ws_bytes, c.used);
    orders[0] = orders[1] = orders[2] = 0;
    *mean_orders = 0.0;
    if (!use_cheb(band)) return GERAF_OK;
    {
        const geraf_status as = smem_attrs(200 * 1024, "shared-memory opt-in", antenna_order_kernel);
        if (as != GERAF_OK) return as;
    }
    launch_cheb_plan(cw, xyz, n, ant_xyz, n_ant, band, st);
    launch_point_order(po, xyz, cw.plan, st);
    gather_xyz<<<grid1d(n, 256), 256, 0, st>>>(xyz, n, po.perm, xyz_p);
    launch_ant_order(ao, ant_xyz, nullptr, n_ant, st);
    cudaError_t e = cudaMemsetAsync(kmax, 0, sizeof(int), st);
    if (e != cudaSuccess) return cuda_status(e, "chebyshev_work");
    group_bbox_kernel<<<n_splits, 256, 0, st>>>(xyz_p, n, per_part, (float)k0_of(band), box);
    split_plan_kernel<<<parts, 256, 0, st>>>(box, ao.rec, n_ant, n_rec, n_ab, ant_per_block, 2.0 * band->df / kC,
                                             band->n_f, CH_TAIL, k0_of(band), cw.plan, splan, rcs, Cs, kmax);
    geraf_status s = check_launch("chebyshev_work");
    if (s != GERAF_OK) return s;
    ChebPlan h;
    std::vector<SplitPlan> hs((size_t)parts);
    int km = 0;
    e = cudaMemcpyAsync(&h, cw.plan, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hs.data(), splan, sizeof(SplitPlan) * parts, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&km, kmax, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e, "chebyshev_work: read back");
    if (!h.run_cheb) return GERAF_OK;
    const int inst = km <= 24 ? 24 : (km <= 32 ? 32 : 64);
    double sum = 0.0;
    for (int g = 0; g < parts; ++g) {
        const int sp = g / n_ab, b = g % n_ab;
        const int64_t j0 = (int64_t)sp * per_part, j1 = std::min<int64_t>(n, j0 + per_part);
        const int64_t a0 = (int64_t)b * ant_per_block, a1 = std::min<int64_t>(n_ant, a0 + ant_per_block);
        const int Kp = hs[g].K;
        const int ex = inst <= 32 ? std::min(inst, Kp <= 8 ? 8 : (Kp + 1) & ~1) : std::max(32, (Kp + 7) / 8 * 8);
        sum += (double)std::max<int64_t>(j1 - j0, 0) * (double)std::max<int64_t>(a1 - a0, 0) * ex;
    }
    orders[0] = h.K;
    orders[1] = km;
    orders[2] = inst;
    *mean_orders = sum / ((double)n * (double)n_ant);
    return GERAF_OK;
}

}  // namespace geraf

// ================================================= render without allocation
// Variant of render for callers that cannot allocate device memory: its
// scratch (packed point tiles, antenna records, split partials) lives in one
// file-scope device array of kNoAllocScratchBytes, which every GPU that loads
// this library holds until the process exits. All calls share the array, so
// calls that overlap on the GPU (other streams, other host threads) race on
// it. Nothing in it must start at zero: every call rewrites all the records
// and partials it later reads. It always runs the per-bin recurrence
// (to_bins_kernel): the Chebyshev form's coefficient tables and moment partials
// (up to hundreds of MiB) do not fit a modest static array, so band->method is
// not consulted.
namespace geraf {
namespace {
constexpr size_t kNoAllocScratchBytes = 32ull << 20;   // 32 MiB
static __device__ __align__(256) unsigned char g_render_scratch[kNoAllocScratchBytes];
std::mutex g_scratch_mu;
void* g_scratch_addr[64];
}  // namespace

geraf_status render_noalloc_impl(const float* xyz, const float* grad, const float* w, const float* t_eff,
                                 int64_t n_pts, const float* ant_xyz, const float* c_ant, int32_t n_ant,
                                 const geraf_band* band, int32_t flags, float* s_out, cudaStream_t st) {
    // once per device, with that device current: the device address of the scratch array
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_status(e, "render_noalloc: cudaGetDevice");
    if (dev < 0 || dev >= 64) return fail(GERAF_ERR_UNSUPPORTED, "render_noalloc: device index %d above 63", dev);
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_scratch_mu);
        if (!g_scratch_addr[dev]) {
            void* p = nullptr;
            e = cudaGetSymbolAddress(&p, g_render_scratch);
            if (e != cudaSuccess) return cuda_status(e, "render_noalloc: cudaGetSymbolAddress");
            g_scratch_addr[dev] = p;
        }
        base = g_scratch_addr[dev];
    }
    BandK bk;
    if (!make_band_k(band, &bk)) return GERAF_ERR_INVALID_ARG;
    ToBinsPlan p = plan_to_bins(n_pts, n_ant, bk.g);
    // fewer point splits when the partials would not fit the static scratch
    WsCarver fixed(nullptr);
    fixed.take<PtRec>((size_t)p.n_tiles * p.TP);
    fixed.take<float4>(p.n_ant_pad);
    const size_t head = align_up(fixed.used, 256);
    const size_t per_split = (size_t)p.n_ant_pad * 32 * p.G * sizeof(float2);
    if (head + per_split > kNoAllocScratchBytes)
        return fail(GERAF_ERR_UNSUPPORTED,
                    "render_noalloc: %lld points x %d antennas x %d bins need %zu bytes of scratch, above the "
                    "%zu-byte static limit (use geraf_render with a caller workspace)",
                    (long long)n_pts, n_ant, band->n_f, head + per_split, kNoAllocScratchBytes);
    const int max_splits = (int)((kNoAllocScratchBytes - head) / per_split);
    if (p.splits > max_splits) {
        p.tiles_per_split = (p.n_tiles + max_splits - 1) / max_splits;
        p.splits = (p.n_tiles + p.tiles_per_split - 1) / p.tiles_per_split;
    }
    WsCarver c(base);
    PtRec* pts = c.take<PtRec>((size_t)p.n_tiles * p.TP);
    float4* ant = c.take<float4>(p.n_ant_pad);
    float2* part = c.take<float2>((size_t)p.splits * p.n_ant_pad * 32 * p.G);
    if (c.used > kNoAllocScratchBytes) return fail(GERAF_ERR_UNSUPPORTED, "render_noalloc: scratch overflow");
    {
        // per device, before anything is launched: a failure leaves nothing in flight
        const geraf_status as = smem_attrs(200 * 1024, "render_noalloc: shared-memory opt-in", to_bins_kernel<false>);
        if (as != GERAF_OK) return as;
    }
    int* err = device_error_word();
    const int64_t n_pad = (int64_t)p.n_tiles * p.TP;
    pack_render_points<<<grid1d(n_pad, 256), 256, 0, st>>>(xyz, grad, w, t_eff, n_pts, n_pad,
                                                           (flags & GERAF_RENDER_DIRECTIONAL) ? 1 : 0, pts);
    pack_antennas<<<grid1d(p.n_ant_pad, 256), 256, 0, st>>>(ant_xyz, c_ant, n_ant, p.n_ant_pad, ant);
    ToBinsArgs a{pts, ant, part, err, p.TP, p.n_tiles, p.tiles_per_split, p.n_ant_pad, p.A_T, bk, nullptr};
    to_bins_kernel<false><<<dim3(p.ant_ctas, p.splits), TB_THREADS, p.smem, st>>>(a);
    reduce_bins<<<grid1d((int64_t)n_ant * band->n_f, 256), 256, 0, st>>>(part, p.splits, n_ant, p.n_ant_pad,
                                                                         band->n_f, 32 * p.G,
                                                                         reinterpret_cast<float2*>(s_out));
    return check_launch("render_noalloc");
}

}  // namespace geraf
