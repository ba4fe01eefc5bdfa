// hi_tp.cu -- the throughput-mode lossless pipeline TCMS1-BIT1-RRE1 of
// cuSZ-Hi (arXiv 2507.11165, Sec. 5.2.3) over a byte sequence (the
// reordered quantization codes), and its inverse.  The paper names the
// stages; the container is this library's reading:
//   stream  = u64 n | u32 chunk | u32 nchunks | u32 size[nchunks] | zero pad
//             to 16 bytes | payloads (each padded to 16 bytes)
//   size[k] = padded payload bytes, bit 31 = chunk stored raw
//   TCMS1   t = (b << 1) ^ (b >> 7), b read as a signed int8
//   BIT1    t zero-padded to m' (m rounded up to 64); plane p = bit 7 - p of
//           every element, element 8 j + b at bit b of the plane's byte j
//   RRE1    bitmap bit i = (v[i] != v[i - 1]), v[-1] = 0, LSB first; kept =
//           the bytes whose bit is set; applied to its own bitmap until a
//           level has at most 64 bytes, which is stored as is
//   payload = top level | kept of the levels below, top down; raw (m bytes)
//             when that would be longer than m.
// Encoding: a CTA per chunk (bit planes by warp ballots, bitmaps by
// ballots, kept bytes placed by per-warp popcount prefixes) into a scratch
// slot per chunk; a scan of the sizes; a gather of the payloads.  Decoding:
// the scan, then a CTA per chunk expanding the levels top down (the byte at
// i is the kept byte of rank popcount(bitmap[0..i])) and transposing the
// bit planes back.
#include "hi_internal.h"
#include "hi_device.cuh"

namespace hi {

constexpr uint32_t kTpChunk = 16384;
constexpr uint32_t kTpRaw = 0x80000000u;
constexpr uint32_t kTpSlot = kTpChunk + 64;  // scratch bytes per chunk (16-byte multiple)
constexpr int kTpThreads = 256;
constexpr int kTpMaxLevels = 6;

__host__ __device__ constexpr uint64_t tp_header_bytes(uint64_t nchunks) { return (16 + 4 * nchunks + 15) / 16 * 16; }

struct TpLevels {
    uint32_t L[kTpMaxLevels];
    int R;  // top level
};

__device__ __forceinline__ TpLevels tp_levels(uint32_t m)
{
    TpLevels T;
    T.L[0] = (m + 63) / 64 * 64;
    T.R = 0;
    while (T.L[T.R] > 64) {
        T.L[T.R + 1] = (T.L[T.R] + 7) / 8;
        ++T.R;
    }
    return T;
}

// Offsets (bytes) of the level buffers in shared memory: level 0 holds m'
// <= kTpChunk bytes, level r > 0 at most kTpChunk / 8^r; each with 64 bytes
// of slack for whole-word bitmap writes.
__host__ __device__ constexpr uint32_t tp_level_off(int r)
{
    uint32_t o = 0, len = kTpChunk;
    for (int k = 0; k < r; ++k) {
        o += (len + 64 + 15) / 16 * 16;
        len /= 8;
    }
    return o;
}
constexpr uint32_t kTpLevelBytes = tp_level_off(kTpMaxLevels);
static_assert(kTpLevelBytes < 20 * 1024, "level buffers");

__device__ __forceinline__ uint8_t tcms1(uint32_t b) { return (uint8_t)((b << 1) ^ ((b & 0x80u) ? 0xffu : 0u)); }
__device__ __forceinline__ uint8_t tcms1_inv(uint32_t t) { return (uint8_t)((t >> 1) ^ ((t & 1u) ? 0xffu : 0u)); }

// Block sum of one value per warp (lane 0's), returned to every thread.
__device__ __forceinline__ uint32_t block_sum_warps(uint32_t v, uint32_t* s_red)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    for (uint32_t w = 0; w < nw; ++w) t += s_red[w];
    __syncthreads();
    return t;
}

// Exclusive prefix (over warps, in warp order) of one value per warp.
__device__ __forceinline__ uint32_t block_prefix_warps(uint32_t v, uint32_t* s_red)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    uint32_t t = 0;
    for (uint32_t w = 0; w < warp; ++w) t += s_red[w];
    __syncthreads();
    return t;
}

// Bits of group g (positions 32 g .. 32 g + 31) that lie below L.
__device__ __forceinline__ uint32_t valid_bits(uint32_t g, uint32_t L)
{
    const uint32_t lo = 32 * g;
    return (L >= lo + 32) ? 0xffffffffu : ((L > lo) ? ((1u << (L - lo)) - 1u) : 0u);
}

// Set bits of the bitmap bm over positions [0, L) (all threads).
__device__ uint32_t bitmap_count(const uint8_t* bm, uint32_t L, uint32_t* s_red)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t* bw = reinterpret_cast<const uint32_t*>(bm);
    uint32_t c = 0;
    for (uint32_t g = warp * 32 + lane; g < (L + 31) / 32; g += nw * 32) c += __popc(bw[g] & valid_bits(g, L));
    c = __reduce_add_sync(0xffffffffu, c);
    return block_sum_warps(c, s_red);
}

// RRE bitmap of v[0..L) into bm (whole words; bits past L are 0); returns
// the number of set bits (all threads).
__device__ uint32_t rre_bitmap(const uint8_t* v, uint32_t L, uint8_t* bm, uint32_t* s_red)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t groups = (L + 31) / 32;
    uint32_t cnt = 0;
    for (uint32_t g = warp; g < groups; g += nw) {
        const uint32_t i = 32 * g + lane;
        const bool f = i < L && v[i] != (i ? v[i - 1] : 0);
        const uint32_t w = __ballot_sync(0xffffffffu, f);
        if (lane == 0) reinterpret_cast<uint32_t*>(bm)[g] = w;
        cnt += __popc(w);
    }
    return block_sum_warps(cnt, s_red);
}

// Each warp's contiguous share of the groups of 32 positions.
__device__ __forceinline__ void warp_groups(uint32_t groups, uint32_t* g0, uint32_t* g1)
{
    const uint32_t warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const uint32_t per = (groups + nw - 1) / nw;
    *g0 = min(warp * per, groups);
    *g1 = min(*g0 + per, groups);
}

// The kept bytes of v (bitmap bm) in order to dst (global).
__device__ void rre_compact(const uint8_t* v, uint32_t L, const uint8_t* bm, uint8_t* __restrict__ dst,
                            uint32_t* s_red)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t* bw = reinterpret_cast<const uint32_t*>(bm);
    uint32_t g0, g1;
    warp_groups((L + 31) / 32, &g0, &g1);
    uint32_t c = 0;
    for (uint32_t g = g0; g < g1; ++g) c += __popc(bw[g] & valid_bits(g, L));
    uint32_t base = block_prefix_warps(c, s_red);
    for (uint32_t g = g0; g < g1; ++g) {
        const uint32_t w = bw[g] & valid_bits(g, L);
        if ((w >> lane) & 1u) dst[base + __popc(w & ((1u << lane) - 1u))] = v[32 * g + lane];
        base += __popc(w);
    }
}

// v[0..L) from its bitmap bm and kept bytes src[0..):  v[i] = the kept byte of
// rank popcount(bm[0..i]), 0 before the first.
__device__ void rre_expand(uint8_t* v, uint32_t L, const uint8_t* bm, const uint8_t* src, uint32_t* s_red)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint32_t* bw = reinterpret_cast<const uint32_t*>(bm);
    uint32_t g0, g1;
    warp_groups((L + 31) / 32, &g0, &g1);
    uint32_t c = 0;
    for (uint32_t g = g0; g < g1; ++g) c += __popc(bw[g] & valid_bits(g, L));
    uint32_t base = block_prefix_warps(c, s_red);
    for (uint32_t g = g0; g < g1; ++g) {
        const uint32_t w = bw[g] & valid_bits(g, L);
        const uint32_t r = base + __popc(w & ((2u << lane) - 1u));
        const uint32_t i = 32 * g + lane;
        if (i < L) v[i] = r ? src[r - 1] : (uint8_t)0;
        base += __popc(w);
    }
}

__global__ void __launch_bounds__(kTpThreads) k_tp_encode_chunks(const uint8_t* __restrict__ in, uint64_t n,
                                                                 uint8_t* __restrict__ slots,
                                                                 uint32_t* __restrict__ sizes, uint32_t nchunks)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ uint32_t s_red[kTpThreads / 32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    for (uint32_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
        const uint8_t* s = in + (uint64_t)k * kTpChunk;
        const uint32_t m = (uint32_t)min((uint64_t)kTpChunk, n - (uint64_t)k * kTpChunk);
        const TpLevels T = tp_levels(m);
        uint8_t* u = tsm + tp_level_off(0);
        const uint32_t pl = T.L[0] / 8;
        // TCMS1 + BIT1: plane p, bytes 4 g .. 4 g + 3 = ballot of bit 7 - p over elements 32 g ..
        for (uint32_t g = warp; g < T.L[0] / 32; g += nw) {
            const uint32_t e = 32 * g + lane;
            const uint32_t t = e < m ? tcms1(s[e]) : 0u;
#pragma unroll
            for (int p = 0; p < 8; ++p) {
                const uint32_t w = __ballot_sync(0xffffffffu, (t >> (7 - p)) & 1u);
                if (lane == (uint32_t)p) reinterpret_cast<uint32_t*>(u + p * pl)[g] = w;
            }
        }
        __syncthreads();
        uint32_t cnt[kTpMaxLevels];
        uint32_t total = 0;
        for (int r = 0; r < T.R; ++r) {
            cnt[r] = rre_bitmap(tsm + tp_level_off(r), T.L[r], tsm + tp_level_off(r + 1), s_red);
            total += cnt[r];
        }
        total += T.L[T.R];
        uint8_t* slot = slots + (uint64_t)k * kTpSlot;
        uint32_t len;
        if (total > m) {
            for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) slot[i] = s[i];
            len = m;
        } else {
            const uint8_t* top = tsm + tp_level_off(T.R);
            for (uint32_t i = threadIdx.x; i < T.L[T.R]; i += blockDim.x) slot[i] = top[i];
            uint32_t off = T.L[T.R];
            for (int r = T.R - 1; r >= 0; --r) {
                rre_compact(tsm + tp_level_off(r), T.L[r], tsm + tp_level_off(r + 1), slot + off, s_red);
                off += cnt[r];
            }
            len = off;
        }
        const uint32_t pad = (len + 15) / 16 * 16;
        for (uint32_t i = len + threadIdx.x; i < pad; i += blockDim.x) slot[i] = 0;
        if (threadIdx.x == 0) sizes[k] = pad | (total > m ? kTpRaw : 0u);
        __syncthreads();  // shared buffers are reused by the next chunk
    }
}

// Exclusive scan of the padded sizes (one CTA): offsets[k] = header +
// sum of sizes before k; with out != nullptr also writes the stream header
// and size table, and the stream length to *len.
__global__ void __launch_bounds__(1024) k_tp_scan(const uint32_t* __restrict__ sizes, uint32_t nchunks, uint64_t n,
                                                  uint64_t* __restrict__ offsets, uint8_t* __restrict__ out,
                                                  uint64_t* __restrict__ len)
{
    __shared__ uint64_t s_part[32];
    __shared__ uint64_t s_base;
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_base = tp_header_bytes(nchunks);
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nchunks; c0 += blockDim.x) {
        const uint32_t k = c0 + threadIdx.x;
        const uint32_t raw = k < nchunks ? sizes[k] : 0u;
        const uint64_t v = raw & ~kTpRaw;
        uint64_t incl = v;
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= (uint32_t)d) incl += t;
        }
        if (lane == 31) s_part[warp] = incl;
        __syncthreads();
        uint64_t before = s_base;
        for (uint32_t w = 0; w < warp; ++w) before += s_part[w];
        if (k < nchunks) {
            offsets[k] = before + incl - v;
            if (out) reinterpret_cast<uint32_t*>(out + 16)[k] = raw;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) {
            uint64_t t = 0;
            for (uint32_t w = 0; w < blockDim.x / 32; ++w) t += s_part[w];
            s_base += t;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0 && out) {
        reinterpret_cast<uint64_t*>(out)[0] = n;
        reinterpret_cast<uint32_t*>(out)[2] = kTpChunk;
        reinterpret_cast<uint32_t*>(out)[3] = nchunks;
        for (uint64_t b = 16 + 4 * (uint64_t)nchunks; b < tp_header_bytes(nchunks); ++b) out[b] = 0;
        *len = s_base;
    }
}

__global__ void __launch_bounds__(256) k_tp_gather(const uint8_t* __restrict__ slots,
                                                   const uint32_t* __restrict__ sizes,
                                                   const uint64_t* __restrict__ offsets, uint32_t nchunks,
                                                   uint8_t* __restrict__ out)
{
    for (uint32_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
        const uint32_t pad = sizes[k] & ~kTpRaw;
        const uint4* src = reinterpret_cast<const uint4*>(slots + (uint64_t)k * kTpSlot);
        uint4* dst = reinterpret_cast<uint4*>(out + offsets[k]);
        for (uint32_t i = threadIdx.x; i < pad / 16; i += blockDim.x) dst[i] = src[i];
    }
}

// Decode, a CTA per chunk; offsets from k_tp_scan over the stream's size
// table.  A stream that does not fit its header, size table or levels sets
// HI_ECORRUPT and leaves those chunks' bytes unwritten.
__global__ void __launch_bounds__(kTpThreads) k_tp_decode_chunks(const uint8_t* __restrict__ in, uint64_t in_len,
                                                                 uint64_t n, uint32_t nchunks,
                                                                 const uint64_t* __restrict__ offsets,
                                                                 uint8_t* __restrict__ out,
                                                                 uint32_t* __restrict__ status)
{
    extern __shared__ __align__(16) unsigned char tsm[];
    __shared__ uint32_t s_red[kTpThreads / 32];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const bool hdr_ok = reinterpret_cast<const uint64_t*>(in)[0] == n &&
                        reinterpret_cast<const uint32_t*>(in)[2] == kTpChunk &&
                        reinterpret_cast<const uint32_t*>(in)[3] == nchunks;
    if (!hdr_ok) {
        if (blockIdx.x == 0 && threadIdx.x == 0) set_status(status, HI_ECORRUPT);
        return;
    }
    uint8_t* pay = tsm + kTpLevelBytes;
    const uint64_t hb = tp_header_bytes(nchunks);
    for (uint32_t k = blockIdx.x; k < nchunks; k += gridDim.x) {
        const uint32_t sz = reinterpret_cast<const uint32_t*>(in + 16)[k];
        const uint32_t pad = sz & ~kTpRaw;
        const bool raw = (sz & kTpRaw) != 0;
        const uint32_t m = (uint32_t)min((uint64_t)kTpChunk, n - (uint64_t)k * kTpChunk);
        const uint64_t off = offsets[k];
        bool ok = pad % 16 == 0 && off % 16 == 0 && pad <= (m + 15) / 16 * 16 && off >= hb && off + pad <= in_len;
        if (raw) ok = ok && pad >= m;
        uint8_t* o = out + (uint64_t)k * kTpChunk;
        if (!ok) {
            if (threadIdx.x == 0) set_status(status, HI_ECORRUPT);
            continue;
        }
        const uint8_t* p = in + off;
        if (raw) {
            for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) o[i] = p[i];
            continue;
        }
        for (uint32_t i = threadIdx.x; i < pad / 16; i += blockDim.x)
            reinterpret_cast<uint4*>(pay)[i] = reinterpret_cast<const uint4*>(p)[i];
        const TpLevels T = tp_levels(m);
        uint8_t* top = tsm + tp_level_off(T.R);
        if (T.L[T.R] > pad) {
            if (threadIdx.x == 0) set_status(status, HI_ECORRUPT);
            __syncthreads();
            continue;
        }
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < T.L[T.R]; i += blockDim.x) top[i] = pay[i];
        __syncthreads();
        uint32_t q = T.L[T.R];
        bool good = true;
        for (int r = T.R - 1; r >= 0; --r) {
            const uint8_t* bm = tsm + tp_level_off(r + 1);
            const uint32_t c = bitmap_count(bm, T.L[r], s_red);
            if (q + c > pad) {
                good = false;
                break;
            }
            rre_expand(tsm + tp_level_off(r), T.L[r], bm, pay + q, s_red);
            q += c;
            __syncthreads();
        }
        if (!good) {
            if (threadIdx.x == 0) set_status(status, HI_ECORRUPT);
            __syncthreads();
            continue;
        }
        // bit planes back to bytes, then magnitude-sign back to two's complement
        const uint8_t* u = tsm + tp_level_off(0);
        const uint32_t pl = T.L[0] / 8;
        for (uint32_t g = warp; g < T.L[0] / 32; g += nw) {
            uint32_t t = 0;
#pragma unroll
            for (int pp = 0; pp < 8; ++pp)
                t |= ((reinterpret_cast<const uint32_t*>(u + pp * pl)[g] >> lane) & 1u) << (7 - pp);
            const uint32_t e = 32 * g + lane;
            if (e < m) o[e] = tcms1_inv(t);
        }
        __syncthreads();
    }
}

size_t tp_ws_bytes(uint64_t n)
{
    const uint64_t nc = (n + kTpChunk - 1) / kTpChunk;
    return (size_t)((4 * nc + 15) / 16 * 16 + 8 * nc + nc * kTpSlot + 16);
}

uint64_t tp_stream_bound(uint64_t n)
{
    const uint64_t nc = (n + kTpChunk - 1) / kTpChunk;
    return tp_header_bytes(nc) + nc * 16 + n + 15;
}

static int tp_grid(uint32_t nchunks, int num_sms)
{
    const uint32_t cap = (uint32_t)num_sms * 4;
    return (int)(nchunks < cap ? (nchunks ? nchunks : 1) : cap);
}

cudaError_t launch_tp_encode(const uint8_t* in, uint64_t n, uint8_t* out, uint64_t* len, void* ws, int num_sms,
                             cudaStream_t st)
{
    const uint32_t nc = (uint32_t)((n + kTpChunk - 1) / kTpChunk);
    uint8_t* w = static_cast<uint8_t*>(ws);
    uint32_t* sizes = reinterpret_cast<uint32_t*>(w);
    uint64_t* offsets = reinterpret_cast<uint64_t*>(w + (4 * (uint64_t)nc + 15) / 16 * 16);
    uint8_t* slots = reinterpret_cast<uint8_t*>(offsets + nc);
    slots = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(slots) + 15) & ~(uintptr_t)15);
    if (nc) {
        k_tp_encode_chunks<<<tp_grid(nc, num_sms), kTpThreads, kTpLevelBytes, st>>>(in, n, slots, sizes, nc);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    k_tp_scan<<<1, 1024, 0, st>>>(sizes, nc, n, offsets, out, len);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !nc) return e;
    k_tp_gather<<<tp_grid(nc, num_sms), 256, 0, st>>>(slots, sizes, offsets, nc, out);
    return cudaGetLastError();
}

cudaError_t launch_tp_decode(const uint8_t* in, uint64_t in_len, uint64_t n, uint8_t* out, uint32_t* status, void* ws,
                             int num_sms, cudaStream_t st)
{
    const uint32_t nc = (uint32_t)((n + kTpChunk - 1) / kTpChunk);
    if (!nc) return cudaSuccess;
    uint64_t* offsets = static_cast<uint64_t*>(ws);
    k_tp_scan<<<1, 1024, 0, st>>>(reinterpret_cast<const uint32_t*>(in + 16), nc, n, offsets, nullptr, nullptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_tp_decode_chunks<<<tp_grid(nc, num_sms), kTpThreads, kTpLevelBytes + kTpChunk, st>>>(in, in_len, n, nc, offsets,
                                                                                          out, status);
    return cudaGetLastError();
}

}  // namespace hi
