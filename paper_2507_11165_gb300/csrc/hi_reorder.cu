// hi_reorder.cu -- quantization-code reordering (cuSZ-Hi, arXiv 2507.11165,
// Sec. 5.2.2, Eq. 3) and its inverse.  The code of the point (x, y, z) (x
// slowest) moves to position I(x, y, z) of a 1D sequence in which each
// interpolation level's codes lie together, coarsest first (the anchors at
// the front), row-major within a level.  The level of a point is the largest
// l <= log2 A with 2^l dividing x, y and z; prefix(l) points precede level l.
// Within level l < log2 A the rank is Eq. 3's row-major index minus the
// all-even points before the point, taken on the stride-2^l subgrid
// (coordinates x >> l, ...; dims the number of multiples of 2^l per dim);
// the anchors are ranked row-major on the anchor grid.
//
// One warp per segment of up to kSeg points of a row, one lane per point:
// the row-major side is read or written 32 consecutive bytes per warp
// access, and so is the sequence side wherever the row's positions run
// consecutively (every row with an odd x or y, and the odd z of the rest).
#include "hi_internal.h"

namespace hi {

constexpr uint32_t kSeg = 1024;

__device__ __forceinline__ uint32_t half_up(uint32_t v) { return (v + 1) >> 1; }

// Position of (x, y, z) in the sequence.
__device__ __forceinline__ uint32_t reorder_pos(const ReorderGeo& G, uint32_t x, uint32_t y, uint32_t z)
{
    const uint32_t v = x | y | z;
    int l = v ? __ffs((int)v) - 1 : G.L;
    if (l > G.L) l = G.L;
    const uint32_t xs = x >> l, ys = y >> l, zs = z >> l;
    uint32_t r = (xs * G.D1[l] + ys) * G.D2[l] + zs;
    if (l < G.L) {
        uint32_t before = half_up(xs) * G.H1[l] * G.H2[l];  // all-even points of the planes before
        if ((xs & 1u) == 0) {
            before += half_up(ys) * G.H2[l];                  // ... of the rows before in this plane
            if ((ys & 1u) == 0) before += half_up(zs);         // ... before in this row
        }
        r -= before;
    }
    return G.prefix[l] + r;
}

// INV = false: seq[I(p)] = codes[p];  INV = true: codes[p] = seq[I(p)].
template <bool INV>
__global__ void __launch_bounds__(256) k_reorder(const uint8_t* __restrict__ src, uint8_t* __restrict__ dst,
                                                 const ReorderGeo G)
{
    const uint32_t lane = threadIdx.x & 31u;
    const uint64_t warp = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t items = (uint64_t)G.n0 * G.n1 * G.segs;
    for (uint64_t it = warp; it < items; it += nwarps) {
        const uint32_t row = (uint32_t)(it / G.segs), seg = (uint32_t)(it - (uint64_t)row * G.segs);
        const uint32_t x = row / G.n1, y = row - x * G.n1;
        const uint32_t z0 = seg * kSeg, z1 = min(z0 + kSeg, G.n2);
        const uint32_t p_row = row * G.n2;
        if ((x | y) & 1u) {
            // the whole row is on the finest level, at consecutive positions
            uint32_t base = G.prefix[0] + (x * G.D1[0] + y) * G.D2[0] - half_up(x) * G.H1[0] * G.H2[0];
            if ((x & 1u) == 0) base -= half_up(y) * G.H2[0];
            for (uint32_t z = z0 + lane; z < z1; z += 32) {
                if constexpr (INV)
                    dst[p_row + z] = src[base + z];
                else
                    dst[base + z] = src[p_row + z];
            }
        } else {
            for (uint32_t z = z0 + lane; z < z1; z += 32) {
                const uint32_t I = reorder_pos(G, x, y, z);
                if constexpr (INV)
                    dst[p_row + z] = src[I];
                else
                    dst[I] = src[p_row + z];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Rows of 16-byte multiples (both buffers 16-byte aligned): a warp stages a
// row of the row-major side in shared memory and moves it run by run.  The
// points of row (x, y) fall into at most L + 1 runs of consecutive sequence
// positions: on the stride-2^l subgrid (row coordinates xs = x >> l,
// ys = y >> l, points zs in [0, D2[l])), if xs or ys is odd every point of
// the row is on level l, in order; if both are even the odd zs are on level
// l, in order, and the even zs go on to level l + 1; at l = L every point is
// an anchor.  Run j-th position B + j holds row element z = zb + zst * j.
// ---------------------------------------------------------------------------
constexpr uint32_t kRowMax = 4096;  // longest row the staged path takes (bytes)
constexpr int kRowWarps = 8;

struct Run {
    uint32_t B, cnt, zb, zst;
};

// The runs of row (x, y), in level order; returns how many (<= L + 1).
__device__ __forceinline__ int row_runs(const ReorderGeo& G, uint32_t x, uint32_t y, Run* r)
{
    int n = 0;
    for (int l = 0;; ++l) {
        const uint32_t xs = x >> l, ys = y >> l;
        const uint32_t row_rank = (xs * G.D1[l] + ys) * G.D2[l];
        if (l == G.L) {
            r[n++] = Run{G.prefix[l] + row_rank, G.D2[l], 0u, 1u << l};
            return n;
        }
        uint32_t before = half_up(xs) * G.H1[l] * G.H2[l];
        if ((xs & 1u) == 0) before += half_up(ys) * G.H2[l];
        if ((xs | ys) & 1u) {
            r[n++] = Run{G.prefix[l] + row_rank - before, G.D2[l], 0u, 1u << l};
            return n;
        }
        if (G.D2[l] >= 2) r[n++] = Run{G.prefix[l] + row_rank - before, G.D2[l] / 2, 1u << l, 2u << l};
    }
}

// seq[B + j] = row[zb + zst j] for a run: aligned 4-byte words, single bytes
// at the run's ends.  sw: the staged row as words (one word of padding).
__device__ __forceinline__ void run_store(const uint32_t* sw, const uint8_t* sb, uint8_t* __restrict__ seq,
                                          const Run& R, uint32_t lane)
{
    const uint32_t head = min((4u - (R.B & 3u)) & 3u, R.cnt);
    const uint32_t nw = (R.cnt - head) >> 2;
    const uint32_t tail0 = head + 4 * nw;
    if (lane < head) seq[R.B + lane] = sb[R.zb + R.zst * lane];
    if (lane < R.cnt - tail0) seq[R.B + tail0 + lane] = sb[R.zb + R.zst * (tail0 + lane)];
    uint32_t* dst = reinterpret_cast<uint32_t*>(seq + R.B + head);
    if (R.zst == 1) {
        for (uint32_t m = lane; m < nw; m += 32) {
            const uint32_t z = R.zb + head + 4 * m;
            dst[m] = __funnelshift_r(sw[z >> 2], sw[(z >> 2) + 1], 8 * (z & 3u));
        }
    } else {
        for (uint32_t m = lane; m < nw; m += 32) {
            const uint32_t z = R.zb + R.zst * (head + 4 * m);
            dst[m] = (uint32_t)sb[z] | ((uint32_t)sb[z + R.zst] << 8) | ((uint32_t)sb[z + 2 * R.zst] << 16) |
                     ((uint32_t)sb[z + 3 * R.zst] << 24);
        }
    }
}

// row[zb + zst j] = seq[B + j] for a run, into the staged row.
__device__ __forceinline__ void run_load(uint8_t* sb, const uint8_t* __restrict__ seq, const Run& R, uint32_t lane)
{
    if (R.zst == 1 && R.zb == 0 && (R.cnt & 3u) == 0) {
        // whole words of the row: each from the two aligned sequence words it straddles
        const uint32_t* sq = reinterpret_cast<const uint32_t*>(seq) + (R.B >> 2);
        const uint32_t sh = 8 * (R.B & 3u);
        uint32_t* sw = reinterpret_cast<uint32_t*>(sb);
        for (uint32_t k = lane; k < (R.cnt >> 2); k += 32) {
            const uint32_t w0 = __ldg(sq + k);
            sw[k] = sh ? __funnelshift_r(w0, __ldg(sq + k + 1), sh) : w0;
        }
        return;
    }
    const uint32_t a0 = R.B & ~3u;  // aligned words covering [B, B + cnt)
    const uint32_t nw = (R.B + R.cnt - a0 + 3) >> 2;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(seq + a0);
    for (uint32_t m = lane; m < nw; m += 32) {
        const uint32_t w = __ldg(src + m);
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const uint32_t j = a0 + 4 * m + t - R.B;  // wraps for bytes before B
            if (j < R.cnt) sb[R.zb + R.zst * j] = (uint8_t)(w >> (8 * t));
        }
    }
}

template <bool INV>
__global__ void __launch_bounds__(kRowWarps * 32) k_reorder_rows(const uint8_t* __restrict__ src,
                                                                uint8_t* __restrict__ dst, const ReorderGeo G)
{
    extern __shared__ __align__(16) unsigned char rsm[];
    const uint32_t lane = threadIdx.x & 31u, wib = threadIdx.x >> 5;
    const uint32_t pitch = G.n2 + 16;  // one word of padding for the funnel shift, 16-byte rows
    uint8_t* sb = rsm + wib * pitch;
    const uint32_t* sw = reinterpret_cast<const uint32_t*>(sb);
    const uint32_t rows = G.n0 * G.n1;
    const uint32_t nv = G.n2 >> 4;
    for (uint32_t row = blockIdx.x * kRowWarps + wib; row < rows; row += gridDim.x * kRowWarps) {
        const uint32_t x = row / G.n1, y = row - x * G.n1;
        Run R[HI_MAX_LEVELS];
        const int nr = row_runs(G, x, y, R);
        if constexpr (!INV) {
            const uint4* s16 = reinterpret_cast<const uint4*>(src + (size_t)row * G.n2);
            for (uint32_t c = lane; c < nv; c += 32) reinterpret_cast<uint4*>(sb)[c] = __ldg(s16 + c);
            __syncwarp();
            for (int k = 0; k < nr; ++k) run_store(sw, sb, dst, R[k], lane);
        } else {
            for (int k = 0; k < nr; ++k) run_load(sb, src, R[k], lane);
            __syncwarp();
            uint4* d16 = reinterpret_cast<uint4*>(dst + (size_t)row * G.n2);
            for (uint32_t c = lane; c < nv; c += 32) d16[c] = reinterpret_cast<const uint4*>(sb)[c];
        }
        __syncwarp();  // the staged row is reused by the next row
    }
}

ReorderGeo make_reorder_geo(const int64_t n[3], int L)
{
    ReorderGeo G{};
    G.n0 = (uint32_t)n[0], G.n1 = (uint32_t)n[1], G.n2 = (uint32_t)n[2];
    G.segs = (G.n2 + kSeg - 1) / kSeg;
    G.L = L;
    uint32_t sub[3] = {G.n0, G.n1, G.n2};
    for (int l = 0; l <= L; ++l) {
        G.D1[l] = sub[1], G.D2[l] = sub[2];
        G.H1[l] = (sub[1] + 1) / 2, G.H2[l] = (sub[2] + 1) / 2;
        // coarser than l: the points whose coordinates are multiples of 2^(l+1)
        G.prefix[l] = (l < L) ? ((sub[0] + 1) / 2) * G.H1[l] * G.H2[l] : 0u;
        for (int d = 0; d < 3; ++d) sub[d] = (sub[d] + 1) / 2;
    }
    return G;
}

cudaError_t launch_reorder(const ReorderGeo& G, const uint8_t* src, uint8_t* dst, bool inverse, int num_sms,
                           cudaStream_t st)
{
    const bool rows_ok = G.n2 % 16 == 0 && G.n2 <= kRowMax && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
                         (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    if (rows_ok) {
        const uint32_t rows = G.n0 * G.n1;
        const size_t smem = (size_t)kRowWarps * (G.n2 + 16);
        const uint32_t want = (rows + kRowWarps - 1) / kRowWarps;
        const uint32_t cap = (uint32_t)num_sms * 8;
        const int grid = (int)(want < cap ? want : cap);
        if (inverse)
            k_reorder_rows<true><<<grid, kRowWarps * 32, smem, st>>>(src, dst, G);
        else
            k_reorder_rows<false><<<grid, kRowWarps * 32, smem, st>>>(src, dst, G);
        return cudaGetLastError();
    }
    const uint64_t items = (uint64_t)G.n0 * G.n1 * G.segs;
    const uint64_t want = (items + 7) / 8;  // 8 warps per block
    const int grid = (int)(want < (uint64_t)num_sms * 8 ? (want ? want : 1) : (uint64_t)num_sms * 8);
    if (inverse)
        k_reorder<true><<<grid, 256, 0, st>>>(src, dst, G);
    else
        k_reorder<false><<<grid, 256, 0, st>>>(src, dst, G);
    return cudaGetLastError();
}

}  // namespace hi
