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
