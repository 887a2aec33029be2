// Shared device helpers of the GB300 rendering kernels: status reporting,
// double-single (hi + lo FP32 pair) arithmetic, mbarrier waits with a time
// limit, 1-D TMA bulk copies, launch geometry.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/geraf.h"

namespace geraf {

// ---------------------------------------------------------------- host side
void set_error(const char* fmt, ...);
geraf_status fail(geraf_status st, const char* fmt, ...);
geraf_status cuda_status(cudaError_t e, const char* what);
int device_sm_count();

// Opts a kernel in to `bytes` of dynamic shared memory on the current device,
// once per (kernel, device): thread-safe, and the CUDA error of a failed
// attempt is returned (nothing is recorded then, so a later call retries).
geraf_status ensure_smem_attr(const void* func, int bytes, const char* what);
template <class... F>
geraf_status smem_attrs(int bytes, const char* what, F*... funcs) {
    geraf_status st = GERAF_OK;
    ((st = st == GERAF_OK ? ensure_smem_attr(reinterpret_cast<const void*>(funcs), bytes, what) : st), ...);
    return st;
}

// device error word: bit 0 = a bounded wait timed out. Read and cleared by
// geraf_poll_device_error().
int* device_error_word();

constexpr double kC = 299792458.0;   // m/s, exact SI value
constexpr int kBinsPerBlock = 32;    // phasor recurrence re-seeded every 32 bins

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Splits a caller workspace into 256-byte aligned slices.
struct WsCarver {
    char* base;
    size_t used = 0;
    explicit WsCarver(void* p) : base(static_cast<char*>(p)) {}
    template <class T> T* take(size_t count) {
        used = align_up(used, 256);
        T* p = base ? reinterpret_cast<T*>(base + used) : nullptr;
        used += count * sizeof(T);
        return p;
    }
};

// Per-band constants: K_b = 2 f_{32 b} / c split into FP32 hi + lo (cycles per
// metre at the first frequency of bin block b) and Kd = 2 df / c.
struct BandK {
    float k[2 * 64];
    float kd;
    int g;          // number of 32-bin blocks
};
bool make_band_k(const geraf_band* band, BandK* out);

// ---------------------------------------------------------------- device side
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Range r = |p - q| as a double-single pair (rh + rl), from FP32 coordinates
// taken as exact. Also returns the FP32 difference vector and rsqrt(r^2).
struct Range {
    float dx, dy, dz;   // rounded differences
    float rh, rl;       // r = rh + rl to ~2^-44 relative
    float rs;           // ~1 / r
};

__device__ __forceinline__ Range pair_range(float px, float py, float pz,
                                            float qx, float qy, float qz) {
    Range R;
    float lx, ly, lz;
    two_sum(px, -qx, R.dx, lx);
    two_sum(py, -qy, R.dy, ly);
    two_sum(pz, -qz, R.dz, lz);
    // squares as hi + lo
    float sx = __fmul_rn(R.dx, R.dx), ex = __fmaf_rn(R.dx, R.dx, -sx);
    float sy = __fmul_rn(R.dy, R.dy), ey = __fmaf_rn(R.dy, R.dy, -sy);
    float sz = __fmul_rn(R.dz, R.dz), ez = __fmaf_rn(R.dz, R.dz, -sz);
    ex = __fmaf_rn(2.0f * R.dx, lx, ex);
    ey = __fmaf_rn(2.0f * R.dy, ly, ey);
    ez = __fmaf_rn(2.0f * R.dz, lz, ez);
    float s12, t12, S, t3;
    two_sum(sx, sy, s12, t12);
    two_sum(s12, sz, S, t3);
    float lo = __fadd_rn(__fadd_rn(__fadd_rn(ex, ey), __fadd_rn(ez, t12)), t3);
    S = fmaxf(S, 1e-30f);
    float rs = rsqrtf(S);
    float r0 = __fmul_rn(S, rs);
    // one Newton step on the double-single square
    float resid = __fadd_rn(__fmaf_rn(-r0, r0, S), lo);
    R.rh = r0;
    R.rl = __fmul_rn(resid, __fmul_rn(0.5f, rs));
    R.rs = rs;
    return R;
}

// Coordinate split of the Chebyshev phasor kernels: x = h + l exactly, with h
// on the 2^-10 m grid and |l| <= 2^-11 m. Differences of two h are exact in
// FP32, and so is the sum of their three squares (multiples of 2^-20 below
// 16 m^2) while every axis difference is below 2 m; the kernels' plan falls
// back to the exact recurrence kernels beyond that.
constexpr float kSplitScale = 1024.0f;
__device__ __forceinline__ void split_coord(float x, float& h, float& l) {
    h = __fmul_rn(rintf(__fmul_rn(x, kSplitScale)), 1.0f / kSplitScale);
    l = __fsub_rn(x, h);
}

// Coordinate split in carrier cycles (the Chebyshev kernels): X = K0 x with
// K0 = 2 f_c / c cycles per metre at the band centre f_c (FP64 product of the
// FP32 coordinate),
// X = h + l with h on the half-cycle grid (exact in FP32 below 2^22 cycles)
// and l the FP32 rounding of the remainder (|l| <= 1/4 cycle, about 0.5 mm).
// Differences of two h are exact, and so is the sum of their three squares
// (multiples of 1/4 below 3 * 2^20) while every axis difference is below 1024
// cycles (about 1.94 m at 79 GHz); the kernels' plan falls back to the exact
// recurrence kernels beyond that. A range in cycles makes the carrier phase
// its fractional part (cyc_frac).
constexpr double kCycGrid = 2.0;
constexpr float kCycAxisMax = 1023.9f;    // cycles: bound on every axis difference
__device__ __forceinline__ void split_cyc(float x, double k0, float& h, float& l) {
    const double X = k0 * (double)x;
    const double hd = rint(X * kCycGrid) * (1.0 / kCycGrid);
    h = (float)hd;
    l = (float)(X - hd);
}

// Fractional part (|.| <= 0.5 + tiny) of a range rh + rl in cycles.
__device__ __forceinline__ float cyc_frac(float rh, float rl) { return __fadd_rn(__fsub_rn(rh, rintf(rh)), rl); }

// Range r = |p - q| as a double-single pair from split coordinates (p = ph +
// pl, q = qh + ql, in metres with the 2^-10 m grid or in cycles with the
// half-cycle grid): with dh = ph - qh (exact) and dl = pl - ql,
//   r^2 = |dh|^2 + sum dl (2 dh + dl),
// the first term exact in FP32 and the second small (|dl| at most one grid
// step), so one Newton step on FP32 sqrt(r^2) gives r to ~1e-10 m (phase
// error < 1e-6 rad at 81 GHz). About 22 instructions against ~53 for pair_range.
__device__ __forceinline__ Range pair_range_split(float pxh, float pyh, float pzh, float pxl, float pyl,
                                                  float pzl, float qxh, float qyh, float qzh, float qxl,
                                                  float qyl, float qzl) {
    Range R;
    const float hx = __fsub_rn(pxh, qxh), hy = __fsub_rn(pyh, qyh), hz = __fsub_rn(pzh, qzh);
    const float lx = __fsub_rn(pxl, qxl), ly = __fsub_rn(pyl, qyl), lz = __fsub_rn(pzl, qzl);
    R.dx = __fadd_rn(hx, lx);
    R.dy = __fadd_rn(hy, ly);
    R.dz = __fadd_rn(hz, lz);
    const float Sh = __fmaf_rn(hz, hz, __fmaf_rn(hy, hy, __fmul_rn(hx, hx)));
    const float cross = __fmaf_rn(lx, __fmaf_rn(2.0f, hx, lx),
                                  __fmaf_rn(ly, __fmaf_rn(2.0f, hy, ly), __fmul_rn(lz, __fmaf_rn(2.0f, hz, lz))));
    const float S = fmaxf(__fadd_rn(Sh, cross), 1e-30f);
    const float rs = rsqrtf(S);
    const float r0 = __fmul_rn(S, rs);
    const float resid = __fadd_rn(__fmaf_rn(-r0, r0, Sh), cross);
    R.rh = r0;
    R.rl = __fmul_rn(resid, __fmul_rn(0.5f, rs));
    R.rs = rs;
    return R;
}

// Fractional part (in cycles, |.| <= 0.5 + tiny) of (rh + rl) * (kh + kl).
__device__ __forceinline__ float phase_frac(float rh, float rl, float kh, float kl) {
    float p = __fmul_rn(rh, kh);
    float e = __fmaf_rn(rh, kh, -p);
    e = __fmaf_rn(rh, kl, e);
    e = __fmaf_rn(rl, kh, e);
    float n = rintf(p);
    return __fadd_rn(__fsub_rn(p, n), e);
}

// Packed pairs of FP32 values (Blackwell f32x2 arithmetic): one instruction
// applies the same IEEE round-to-nearest operation to both lanes. The lane
// throughput equals scalar FFMA; the gain is half the issue slots per flop.
typedef uint64_t f2;

__device__ __forceinline__ f2 pk2(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(f2 v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// 1-D TMA bulk copy global -> shared, completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void tma_load_1d(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 16-byte asynchronous global -> shared copy (zero-filled when src_bytes = 0)
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
// Hint: bring global [src, src + bytes) into L2 (src 16-byte aligned, bytes a
// multiple of 16, the whole range inside one allocation).
__device__ __forceinline__ void prefetch_l2_bulk(const void* src, uint32_t bytes) {
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\n\tcp.async.wait_group 0;" ::: "memory");
}

__device__ __forceinline__ uint64_t global_timer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Waits for phase `parity` of `bar` for at most ~limit_ns. Returns false on
// timeout (the caller records it and leaves).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns = 2000000000ull) {
    if (mbar_try_wait(bar, parity)) return true;
    uint64_t t0 = global_timer_ns();
    for (uint32_t it = 0; it < (1u << 30); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 63u) == 63u && global_timer_ns() - t0 > limit_ns) return false;
    }
    return false;
}

// After a timed-out wait at iteration `it` of a two-buffer TMA pipeline: give
// the copies still in flight (that iteration's and, if issued, the next one's)
// a bounded time to land before the CTA leaves, since its shared memory is
// handed to the next CTA on the SM.
__device__ __forceinline__ void mbar_drain2(uint64_t* bar, int it, int n_my) {
    mbar_wait(&bar[it & 1], (it >> 1) & 1, 100000000ull);
    if (it + 1 < n_my) mbar_wait(&bar[(it + 1) & 1], ((it + 1) >> 1) & 1, 100000000ull);
}

}  // namespace geraf
