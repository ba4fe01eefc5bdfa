// hi_device.cuh -- device-side building blocks shared by the kernels of the
// interpolation predictor / quantizer (cuSZ-Hi, arXiv 2507.11165).
//
// Everything here is compiled with -fmad=false: every float operation is
// rounded on its own, in the order written, so that the kernels reproduce the
// fixed evaluation order the method's reconstruction depends on (Eq. 1: the
// decompressor must rebuild exactly the values the compressor predicted from).
#pragma once

#include <cstdint>
#include <map>
#include <mutex>
#include <utility>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/hi.h"

namespace hi {

constexpr int kRadius = 128;      // code = q + 128, q in [-127, 127] (Sec. 5.2.1)
constexpr float kQmax = 127.5f;   // |t| must stay below this for a valid code
// Every mbarrier wait is bounded by wall-clock time: it gives up after
// kWaitLimitNs of the global nanosecond timer.  Each try_wait may suspend the
// thread for up to kSuspendNs instead of spinning.  kSpinLimit is a second,
// iteration-count bound, kept far above what a healthy wait needs.
constexpr uint32_t kSpinLimit = 1u << 30;
constexpr uint32_t kSuspendNs = 100000;
constexpr uint64_t kWaitLimitNs = 2000000000ull;

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Raise a kernel's dynamic shared-memory limit to at least smem on the
// current device; the runtime is asked only when a larger value is needed.
template <typename K>
static cudaError_t set_max_smem(K kern, size_t smem)
{
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> done;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    std::lock_guard<std::mutex> lock(mu);
    size_t& have = done[{dev, reinterpret_cast<const void*>(kern)}];
    if (have >= smem) return cudaSuccess;
    err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err == cudaSuccess) have = smem;
    return err;
}

// Block geometry for anchor stride A (Sec. 5.1.1): (A+1) points per active
// dim.  Shared-memory tiles keep the field's row-major order with the fastest
// dim padded so that every row starts on a 16-byte boundary (the unit a TMA
// box row is written in).
template <int A>
struct TileGeom {
    static constexpr int P = A + 1;
    static constexpr int L = (A == 2) ? 1 : (A == 4) ? 2 : (A == 8) ? 3 : (A == 16) ? 4 : 5;
    static constexpr int PX = (P + 3) / 4 * 4;     // float pitch of dim 2
    static constexpr int PY = P * PX;              // float pitch of dim 0 (dim 1 pitch = PX)
    // byte pitch of dim 2 for codes: an odd number of 16-byte chunks, so that
    // 16-byte accesses to consecutive rows hit distinct banks
    static constexpr int CX = ((P + 15) / 16 % 2 == 1) ? (P + 15) / 16 * 16 : (P + 15) / 16 * 16 + 16;
    static constexpr int CY = P * CX;              // byte pitch of dim 0 for codes
};

// Geometry of a field, passed by value to every kernel.
struct FieldGeo {
    int64_t n[3];   // dims, slowest -> fastest
    int nb[3];      // blocks per dim
    int na[3];      // anchors per dim
    int64_t N;      // points
    int ntiles;     // nb0 * nb1 * nb2
    int b0;         // planes of a tile along dim 0 in shared memory: A+1, or 1 if n0 == 1
    int ni[3];      // queue order: tiles with t_d < ni_d for all d (whole tiles) come first
};

// ---------------------------------------------------------------------------
// Stencils (Sec. 5.1.2) -- a = f(c-3s), b = f(c-s), u = f(c+s), v = f(c+3s).
// Lagrange midpoint weights: linear (1,1)/2, cubic (-1,9,9,-1)/16, one-sided
// quadratics (3,6,-1)/8 and (-1,6,3)/8; with no right neighbour (global
// upper edge only) linear extrapolation (3b - a)/2, else a copy of b.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float predict(bool cubic, bool have_l3, bool have_r, bool have_r3, float a, float b,
                                         float u, float v)
{
    if (!have_r) return have_l3 ? __fmul_rn(__fsub_rn(__fmul_rn(3.0f, b), a), 0.5f) : b;
    if (!cubic) return __fmul_rn(__fadd_rn(b, u), 0.5f);
    if (have_l3 && have_r3)
        return __fmul_rn(__fsub_rn(__fmul_rn(9.0f, __fadd_rn(b, u)), __fadd_rn(a, v)), 0.0625f);
    if (have_r3) return __fmul_rn(__fsub_rn(__fadd_rn(__fmul_rn(3.0f, b), __fmul_rn(6.0f, u)), v), 0.125f);
    if (have_l3) return __fmul_rn(__fsub_rn(__fadd_rn(__fmul_rn(6.0f, b), __fmul_rn(3.0f, u)), a), 0.125f);
    return __fmul_rn(__fadd_rn(b, u), 0.5f);
}

// Rounding to an integer without a conversion instruction: for |t| < 2^22,
// fl(t + M) with M in [2^23, 2^24) has unit spacing, so the addition rounds t
// to the nearest integer; with M even the tie goes to the even integer,
// exactly as rint.  That integer is the sum's low mantissa bits, and
// fl(sum - M) is it as a float.  The quantizer takes M = 1.5 * 2^23 + 128,
// whose bit pattern ends in 0x80: the low byte of the sum's bit pattern is
// then q + 128, the code itself.  (Larger |t| only occur for outliers, whose
// code and value do not use the result.)
constexpr float kRoundMagic = 12582912.0f;   // 1.5 * 2^23
constexpr float kRoundMagicQ = 12583040.0f;  // 1.5 * 2^23 + 128
constexpr int kRoundMagicBits = 0x4B400000;

// Linear quantization (Sec. 5.2.1): returns the code in its low byte (0 =
// outlier) and the reconstructed value.  t = (x - p) * r; q = rint(t) (ties
// to even); x' = p + q * 2eps; an outlier when !(|t| < 127.5) or
// !(|x - x'| < eb_f).
__device__ __forceinline__ int quantize(float x, float p, float eb_f, float ebx2_f, float r_f, float& xr_out)
{
    const float t = __fmul_rn(__fsub_rn(x, p), r_f);
    const float m = __fadd_rn(t, kRoundMagicQ);
    const float qf = __fsub_rn(m, kRoundMagicQ);  // rint(t)
    const float xr = __fadd_rn(p, __fmul_rn(qf, ebx2_f));
    const bool ok = (fabsf(t) < kQmax) && (fabsf(__fsub_rn(x, xr)) < eb_f);
    xr_out = ok ? xr : x;
    return ok ? __float_as_int(m) : 0;  // low byte: q + 128
}

__device__ __forceinline__ float dequantize(int code, float p, float ebx2_f)
{
    // (float)(code - 128), exactly, through the same constant
    const float qf = __fsub_rn(__int_as_float(code + (kRoundMagicBits - kRadius)), kRoundMagic);
    return __fadd_rn(p, __fmul_rn(qf, ebx2_f));
}

// First error wins.
__device__ __forceinline__ void set_status(uint32_t* status, uint32_t code)
{
    // first error wins; once one is recorded, later callers only read
    if (status && *reinterpret_cast<volatile uint32_t*>(status) == 0u) atomicCAS(status, 0u, code);
}

// ---------------------------------------------------------------------------
// mbarrier + TMA (inline PTX, sm_90+ forms that sm_103a keeps)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(mbar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// 4-byte asynchronous global -> shared copy (no register round trip, many in
// flight per thread); cp_async_wait_all waits for the calling thread's copies.
__device__ __forceinline__ void cp_async4(void* dst, const void* src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async16(void* dst, const void* src)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* mbar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes)
                 : "memory");
}

// Bounded wait on the given phase parity; false when the bound ran out
// (limit_ns of the global timer, or `limit` polls).
__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, uint32_t limit,
                                          uint64_t limit_ns = kWaitLimitNs)
{
    const uint32_t a = smem_addr(mbar);
    uint64_t t0 = 0;
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(a), "r"(parity), "r"(kSuspendNs)
            : "memory");
        if (done) return true;
        if (it == 0) {
            t0 = global_ns();
        } else if ((it & 15) == 0 && global_ns() - t0 > limit_ns) {
            return false;
        }
    }
    return false;
}

// After a wait gave up: a bulk copy issued on this barrier may still write
// into the CTA's shared memory, so the CTA stays until the phase completes,
// bounded by ten times the usual limit (past that the copy engine is not
// answering and nothing the kernel does can make the memory safe).
__device__ __forceinline__ void drain_wait(uint64_t* mbar, uint32_t parity)
{
    (void)mbar_wait(mbar, parity, kSpinLimit, 10 * kWaitLimitNs);
}

// 3D tiled TMA load of one box into shared memory, completing on mbar.
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z, uint64_t* mbar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(mbar))
        : "memory");
}

// Pull one box of the tensor into L2 (no shared memory, no completion).
__device__ __forceinline__ void tma_prefetch_3d(const CUtensorMap* map, int x, int y, int z)
{
    asm volatile("cp.async.bulk.prefetch.tensor.3d.L2.global.tile [%0, {%1, %2, %3}];" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(z)
                 : "memory");
}

// Pull the cache line holding p into L2.
__device__ __forceinline__ void prefetch_l2(const void* p)
{
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// Tile coordinates of a row-major block id.
__device__ __forceinline__ void tile_coords_rm(const FieldGeo& g, int tile, int t[3])
{
    t[2] = tile % g.nb[2];
    const int r = tile / g.nb[2];
    t[1] = r % g.nb[1];
    t[0] = r / g.nb[1];
}

// Tile coordinates of queue position `pos`: the ni0 x ni1 x ni2 interior
// tiles in row-major order first, then the tiles of the upper faces (the
// field's edge tiles when its extent is not a multiple of A), face by face.
// With ni = nb this is plain row-major order over the block grid.
__device__ __forceinline__ void tile_coords(const FieldGeo& g, int pos, int t[3])
{
    const int n_int = g.ni[0] * g.ni[1] * g.ni[2];
    if (pos < n_int) {
        t[2] = pos % g.ni[2];
        const int r = pos / g.ni[2];
        t[1] = r % g.ni[1];
        t[0] = r / g.ni[1];
        return;
    }
    int q = pos - n_int;
    if (g.ni[0] < g.nb[0]) {  // face t0 = nb0 - 1: nb1 x nb2 tiles
        const int n = g.nb[1] * g.nb[2];
        if (q < n) {
            t[0] = g.nb[0] - 1, t[1] = q / g.nb[2], t[2] = q % g.nb[2];
            return;
        }
        q -= n;
    }
    if (g.ni[1] < g.nb[1]) {  // face t1 = nb1 - 1, t0 < ni0: ni0 x nb2 tiles
        const int n = g.ni[0] * g.nb[2];
        if (q < n) {
            t[1] = g.nb[1] - 1, t[0] = q / g.nb[2], t[2] = q % g.nb[2];
            return;
        }
        q -= n;
    }
    // face t2 = nb2 - 1, t0 < ni0, t1 < ni1
    t[2] = g.nb[2] - 1, t[0] = q / g.ni[1], t[1] = q % g.ni[1];
}

}  // namespace hi
