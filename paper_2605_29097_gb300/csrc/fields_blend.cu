// Lensless sampling, analytic fields and lensless alpha blending (+ adjoint).
// These steps touch each point a handful of times and are bound by HBM
// bandwidth: one thread per point (sampling, fields) or per primary column
// (blending, whose depth scan is sequential); depth-major storage makes every
// load and store of a warp coalesced.
#include <math.h>

#include "common.cuh"

namespace geraf {

namespace {

// ----------------------------------------------------------------- sampling
// SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number k of seed.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t k) {
    uint64_t z = seed + (k + 1ull) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ double uniform01(uint64_t seed, uint64_t step, uint64_t stream, uint64_t index) {
    const uint64_t k = (step << 42) | (stream << 40) | index;
    return (double)(splitmix64(seed, k) >> 11) * 0x1.0p-53;
}

// float(lo + (i + u) * pitch), one FP64 rounding per operation (no contraction)
__device__ __forceinline__ float grid_coord(float lo, int64_t i, double u, float pitch) {
    double t = __dadd_rn((double)i, u);
    t = __dmul_rn(t, (double)pitch);
    return __double2float_rn(__dadd_rn((double)lo, t));
}

__global__ void sample_kernel(geraf_grid g, int mode, uint64_t seed, uint64_t step, float* __restrict__ xyz,
                              float* __restrict__ apr) {
    const int64_t n_ray = (int64_t)g.n[0] * g.n[1];
    const int64_t n = n_ray * g.n[2];
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int64_t ray = j % n_ray, k = j / n_ray;
    const int64_t ix = ray % g.n[0], iy = ray / g.n[0];
    double ux = 0.5, uy = 0.5, uz = 0.5;
    if (mode == GERAF_SAMPLE_STRATIFIED) {
        ux = uniform01(seed, step, 0, (uint64_t)ray);
        uy = uniform01(seed, step, 1, (uint64_t)ray);
        uz = uniform01(seed, step, 2, (uint64_t)j);
    }
    const float x = grid_coord(g.lo[0], ix, ux, g.pitch[0]);
    const float y = grid_coord(g.lo[1], iy, uy, g.pitch[1]);
    xyz[j] = x;
    xyz[n + j] = y;
    xyz[2 * n + j] = grid_coord(g.lo[2], k, uz, g.pitch[2]);
    if (k == 0 && apr) {
        apr[ray] = x;
        apr[n_ray + ray] = y;
        apr[2 * n_ray + ray] = g.aperture_z;
    }
}

// ------------------------------------------------------------ analytic fields
// primitive record: kind, a, c[3], p[3]
__device__ __forceinline__ float prim_sdf(const float* pr, float x, float y, float z, float& gx, float& gy,
                                          float& gz) {
    const int kind = (int)pr[0];
    const float dx = x - pr[2], dy = y - pr[3], dz = z - pr[4];
    if (kind == GERAF_PRIM_SPHERE) {
        const float r = sqrtf(dx * dx + dy * dy + dz * dz);
        const float ir = r > 0.0f ? 1.0f / r : 0.0f;
        gx = dx * ir; gy = dy * ir; gz = dz * ir;
        return r - pr[5];
    }
    if (kind == GERAF_PRIM_BOX) {
        const float qx = fabsf(dx) - pr[5], qy = fabsf(dy) - pr[6], qz = fabsf(dz) - pr[7];
        const float mx = fmaxf(qx, 0.0f), my = fmaxf(qy, 0.0f), mz = fmaxf(qz, 0.0f);
        const float out = sqrtf(mx * mx + my * my + mz * mz);
        const float qmax = fmaxf(qx, fmaxf(qy, qz));
        const float sx = dx >= 0.0f ? 1.0f : -1.0f, sy = dy >= 0.0f ? 1.0f : -1.0f, sz = dz >= 0.0f ? 1.0f : -1.0f;
        if (qmax > 0.0f) {
            const float io = 1.0f / out;
            gx = sx * mx * io; gy = sy * my * io; gz = sz * mz * io;
        } else {
            // gradient of the largest q (first on ties, like argmax)
            gx = gy = gz = 0.0f;
            if (qx >= qy && qx >= qz) gx = sx;
            else if (qy >= qz) gy = sy;
            else gz = sz;
        }
        return out + fminf(qmax, 0.0f);
    }
    if (kind == GERAF_PRIM_ELLIPSOID) {
        const float ex = dx / pr[5], ey = dy / pr[6], ez = dz / pr[7];
        const float k0 = sqrtf(ex * ex + ey * ey + ez * ez);
        const float m = fminf(pr[5], fminf(pr[6], pr[7]));
        const float ik = k0 > 0.0f ? m / k0 : 0.0f;
        gx = ik * dx / (pr[5] * pr[5]); gy = ik * dy / (pr[6] * pr[6]); gz = ik * dz / (pr[7] * pr[7]);
        return (k0 - 1.0f) * m;
    }
    // half-space
    gx = pr[5]; gy = pr[6]; gz = pr[7];
    return dx * pr[5] + dy * pr[6] + dz * pr[7];
}

__global__ void analytic_fields_kernel(const float* __restrict__ prims, int n_prims, const float* __restrict__ xyz,
                                       int64_t n, float* __restrict__ sdf, float* __restrict__ grad,
                                       float* __restrict__ refl) {
    extern __shared__ float sp[];
    for (int i = threadIdx.x; i < 8 * n_prims; i += blockDim.x) sp[i] = prims[i];
    __syncthreads();
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float x = xyz[j], y = xyz[n + j], z = xyz[2 * n + j];
    float best = INFINITY, bx = 0.0f, by = 0.0f, bz = 0.0f, ba = 0.0f;
    for (int k = 0; k < n_prims; ++k) {
        float gx, gy, gz;
        const float f = prim_sdf(sp + 8 * k, x, y, z, gx, gy, gz);
        if (f < best) {
            best = f; bx = gx; by = gy; bz = gz; ba = sp[8 * k + 1];
        }
    }
    sdf[j] = best;
    if (grad) {
        grad[j] = bx;
        grad[n + j] = by;
        grad[2 * n + j] = bz;
    }
    if (refl) refl[j] = ba;
}

// -------------------------------------------------------------------- blend
// accurate 1 - Phi_s(f) = sigma(-s f)
__device__ __forceinline__ float one_minus_cdf(float x) { return 1.0f / (1.0f + expf(x)); }

// Thread = one primary column; the depth scan runs in chunks of BL_CH depths
// whose loads are all issued before the chunk's arithmetic (the scan itself is
// sequential per column, so memory-level parallelism comes from the chunk).
constexpr int BL_CH = 16;
constexpr int BL_THREADS = 64;

__global__ void __launch_bounds__(BL_THREADS) blend_kernel(const float* __restrict__ sdf,
                                                           const float* __restrict__ refl,
                                                           const float* __restrict__ keep, int n_ray, int n_z,
                                                           const float* __restrict__ sdf_apr, float s, float a_tx,
                                                           float* __restrict__ alpha, float* __restrict__ T,
                                                           float* __restrict__ w, float* __restrict__ t_eff) {
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_ray) return;
    const float c_ray = 1.0f / (1.0f + expf(-s * sdf_apr[ray]));
    float Tk = 1.0f;
    float fk = sdf[ray];
    for (int k0 = 0; k0 < n_z; k0 += BL_CH) {
        float fv[BL_CH], av[BL_CH];
#pragma unroll
        for (int q = 0; q < BL_CH; ++q) {
            const int k = k0 + q;
            fv[q] = k + 1 < n_z ? sdf[(size_t)(k + 1) * n_ray + ray] : 0.0f;
            av[q] = k < n_z ? refl[(size_t)k * n_ray + ray] : 0.0f;
            if (keep && k < n_z) av[q] *= keep[(size_t)k * n_ray + ray];
        }
#pragma unroll
        for (int q = 0; q < BL_CH; ++q) {
            const int k = k0 + q;
            if (k >= n_z) break;
            const size_t j = (size_t)k * n_ray + ray;
            float al = 0.0f;
            const float fn = fv[q];
            if (k + 1 < n_z) {
                // alpha = 1 - Phi(f_{k+1}) / Phi(f_k) = -expm1(s (f_{k+1} - f_k)) * sigma(-s f_{k+1})
                if (fn < fk) al = -expm1f(s * (fn - fk)) * one_minus_cdf(s * fn);
            }
            alpha[j] = al;
            T[j] = Tk;
            w[j] = av[q] * al * a_tx;
            t_eff[j] = Tk + c_ray;
            Tk = Tk * (1.0f - al);
            fk = fn;
        }
    }
}

__global__ void cdf_kernel(const float* __restrict__ f, int n, float s, float* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = 1.0f / (1.0f + expf(-s * f[i]));
}

// reverse depth scan; per-ray partials of dL/ds and dL/dA'_tx in `part`
__global__ void __launch_bounds__(BL_THREADS) blend_backward_kernel(
    const float* __restrict__ sdf, const float* __restrict__ refl, const float* __restrict__ keep,
    const float* __restrict__ alpha, const float* __restrict__ T, int n_ray, int n_z, float s, float a_tx,
    const float* __restrict__ d_w,
    const float* __restrict__ d_teff, float* __restrict__ d_sdf, float* __restrict__ d_refl, float2* __restrict__ part) {
    const int ray = blockIdx.x * blockDim.x + threadIdx.x;
    if (ray >= n_ray) return;
    float gT_next = 0.0f;      // total dL/dT_{k+1}
    float carry = 0.0f;        // contribution to d_sdf[k+1] from alpha_{k+1} (left end point)
    float ds = 0.0f, datx = 0.0f;
    float f_next = 0.0f;
    // chunks of BL_CH depths from the top: [k1 - BL_CH + 1, k1], loads first
    for (int k1 = n_z - 1; k1 >= 0; k1 -= BL_CH) {
        float fv[BL_CH], av[BL_CH], alv[BL_CH], tv[BL_CH], dwv[BL_CH], dtv[BL_CH];
#pragma unroll
        for (int q = 0; q < BL_CH; ++q) {
            const int k = k1 - q;
            const bool ok = k >= 0;
            const size_t j = (size_t)(ok ? k : 0) * n_ray + ray;
            fv[q] = ok ? sdf[j] : 0.0f;
            av[q] = ok ? refl[j] : 0.0f;
            alv[q] = ok ? alpha[j] : 0.0f;
            tv[q] = ok ? T[j] : 0.0f;
            dwv[q] = ok && d_w ? d_w[j] : 0.0f;
            if (ok && keep) dwv[q] *= keep[j];     // w = keep a alpha A'_tx: d_w reaches a, alpha, A'_tx through keep
            dtv[q] = ok && d_teff ? d_teff[j] : 0.0f;
        }
#pragma unroll
        for (int q = 0; q < BL_CH; ++q) {
            const int k = k1 - q;
            if (k < 0) break;
            const size_t j = (size_t)k * n_ray + ray;
            const float fk = fv[q], ak = av[q], alk = alv[q], Tk = tv[q];
            const float dwk = dwv[q], dtk = dtv[q];
            float dal = dwk * ak * a_tx;
            d_refl[j] = dwk * alk * a_tx;
            datx += dwk * ak * alk;
            float gT = dtk;
            float right = 0.0f, left = 0.0f;
            if (k + 1 < n_z) {
                dal -= gT_next * Tk;
                gT = dtk + gT_next * (1.0f - alk);
                if (f_next < fk) {
                    const float R = 1.0f - alk;                // Phi_{k+1} / Phi_k
                    const float s0 = one_minus_cdf(s * fk), s1 = one_minus_cdf(s * f_next);
                    left = dal * R * s * s0;
                    right = -dal * R * s * s1;
                    ds += -dal * R * (f_next * s1 - fk * s0);
                }
                d_sdf[j + n_ray] = carry + right;
            }
            carry = left;
            gT_next = gT;
            f_next = fk;
        }
    }
    d_sdf[ray] = carry;
    part[ray] = make_float2(ds, datx);
}

__global__ void reduce_pairs(const float2* __restrict__ part, int n, float* __restrict__ out) {
    __shared__ double r0[256], r1[256];
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        a += part[i].x;
        b += part[i].y;
    }
    r0[threadIdx.x] = a;
    r1[threadIdx.x] = b;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if (threadIdx.x < k) {
            r0[threadIdx.x] += r0[threadIdx.x + k];
            r1[threadIdx.x] += r1[threadIdx.x + k];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        out[0] = (float)r0[0];
        out[1] = (float)r1[0];
    }
}

inline unsigned grid1d(int64_t n, int b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

geraf_status sample_impl(const geraf_grid* g, int32_t mode, uint64_t seed, uint64_t step, float* xyz, float* apr,
                         cudaStream_t st) {
    const int64_t n = (int64_t)g->n[0] * g->n[1] * g->n[2];
    sample_kernel<<<grid1d(n, 256), 256, 0, st>>>(*g, mode, seed, step, xyz, apr);
    return cuda_status(cudaGetLastError(), "sample");
}

geraf_status analytic_fields_impl(const float* prims, int n_prims, const float* xyz, int64_t n, float* sdf,
                                  float* grad, float* refl, cudaStream_t st) {
    analytic_fields_kernel<<<grid1d(n, 256), 256, 8 * n_prims * sizeof(float), st>>>(prims, n_prims, xyz, n, sdf,
                                                                                    grad, refl);
    return cuda_status(cudaGetLastError(), "fields(analytic)");
}

geraf_status blend_impl(const float* sdf, const float* refl, const float* keep, int32_t n_ray, int32_t n_z,
                        const float* sdf_apr, const float* sdf_ant, int32_t n_ant, float s, float a_tx, float* alpha,
                        float* T, float* w, float* t_eff, float* c_ant, cudaStream_t st) {
    blend_kernel<<<grid1d(n_ray, BL_THREADS), BL_THREADS, 0, st>>>(sdf, refl, keep, n_ray, n_z, sdf_apr, s, a_tx,
                                                                     alpha, T, w, t_eff);
    if (n_ant > 0) cdf_kernel<<<grid1d(n_ant, 256), 256, 0, st>>>(sdf_ant, n_ant, s, c_ant);
    return cuda_status(cudaGetLastError(), "blend");
}

geraf_status blend_backward_impl(const float* sdf, const float* refl, const float* keep, const float* alpha,
                                 const float* T, int32_t n_ray, int32_t n_z, float s, float a_tx, const float* d_w,
                                 const float* d_teff, float* d_sdf, float* d_refl, float* d_scalars, void* ws,
                                 size_t* ws_bytes, cudaStream_t st) {
    WsCarver c(ws);
    float2* part = c.take<float2>(n_ray);
    if (!ws) { *ws_bytes = c.used; return GERAF_OK; }
    if (*ws_bytes < c.used)
        return fail(GERAF_ERR_WORKSPACE, "blend_backward: workspace %zu < %zu bytes", *ws_bytes, c.used);
    blend_backward_kernel<<<grid1d(n_ray, BL_THREADS), BL_THREADS, 0, st>>>(sdf, refl, keep, alpha, T, n_ray, n_z,
                                                                           s, a_tx, d_w, d_teff, d_sdf, d_refl, part);
    reduce_pairs<<<1, 256, 0, st>>>(part, n_ray, d_scalars);
    return cuda_status(cudaGetLastError(), "blend_backward");
}

}  // namespace geraf
