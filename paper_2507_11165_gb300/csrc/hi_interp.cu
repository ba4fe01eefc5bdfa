// hi_interp.cu -- fused interpolation-predict + quantize kernel and its
// inverse, the level-by-level reconstruction (cuSZ-Hi, arXiv 2507.11165,
// Sec. 3.2, Sec. 5.1.1-5.1.2, Sec. 5.2.1).
//
// Persistent CTAs take blocks ("tiles") of (A+1)^d points from a queue in
// ascending order.  A tile is staged in shared memory by one 3D TMA box load
// (plain loads when the field's strides do not meet the TMA rules); with two
// tile buffers the next tile's load is in flight while the current one is
// processed.  Every level (stride S = A/2 .. 1) runs its three 1D passes in
// the configured dimension sequence; predictions read values already
// reconstructed in shared memory (closed loop), so the decompressor repeats
// exactly the same arithmetic.
//
// Pass geometry is compile-time wherever possible: every (level, spline,
// pass dimension) is its own instantiation.
//   * full 3D tiles (extent A in every dim, A = 8 or 16) -- the bulk of any
//     large field -- also fix the dimension sequence at compile time, so line
//     counts, stencil cases and shared-memory offsets are constants;
//   * all other tiles (ragged field edges, 1D/2D fields, other A) take the
//     extents at run time.
// Passes along the contiguous dim move whole rows with 16-byte shared-memory
// accesses (conflict-free at the 16-byte-multiple, odd-word row pitch);
// passes along the other dims give each thread one line, lanes adjacent along
// the contiguous dim.
//
// Shared faces between tiles are computed by both tiles with identical
// results; only the owning tile (the one with the lower block index, or the
// last block for the field's upper face) writes codes, histogram counts,
// outliers and reconstructed values.  Codes are staged in shared memory and
// leave the tile in its epilogue, which also finds the outliers (code 0) and
// counts the histogram.
#include <cstdint>

#include "hi_device.cuh"
#include "hi_internal.h"

namespace hi {

constexpr int kMaxThreads = 256;

// Shared-memory layouts of one tile (planes b0 = A+1, or 1 for 1D/2D fields).
template <int A>
struct Lay {
    using TG = TileGeom<A>;
    static constexpr int P = A + 1;
    static constexpr int PX = TG::PX;   // floats per row (16-byte multiple)
    static constexpr int PY = P * PX;   // floats per plane
    static constexpr int CXC = PX;      // compress code staging: bytes per row
    static constexpr int CYC = P * CXC;
    static constexpr int CXD = TG::CX;  // decompress codes (TMA box rows, 16-byte multiple)
    static constexpr int CYD = P * CXD;
};

__host__ __device__ constexpr int round128(int b) { return (b + 127) / 128 * 128; }

template <int A>
__host__ __device__ constexpr int vbuf_bytes(int b0)
{
    return round128(b0 * Lay<A>::P * Lay<A>::PX * 4);
}

struct TileInfo {
    int o[3];    // origin (global coords)
    int e[3];    // extent: last local coordinate per dim (0 for inactive dims)
    int own[3];  // last owned local coordinate per dim
};

template <int A>
__device__ __forceinline__ TileInfo tile_info(const FieldGeo& g, int tile)
{
    TileInfo ti;
    int t[3];
    tile_coords(g, tile, t);
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        ti.o[d] = t[d] * A;
        const int rem = (int)(g.n[d] - 1 - ti.o[d]);
        ti.e[d] = (g.n[d] == 1) ? 0 : (rem < A ? rem : A);
        ti.own[d] = (t[d] == g.nb[d] - 1) ? ti.e[d] : A - 1;
    }
    return ti;
}

// Global linear index of a float offset in the tile buffer.
template <int A>
__device__ __forceinline__ int64_t global_index(const FieldGeo& g, const int o[3], int vi)
{
    constexpr int PY = Lay<A>::PY, PX = Lay<A>::PX;
    const int c0 = vi / PY;
    const int rem = vi - c0 * PY;
    const int c1 = rem / PX;
    const int c2 = rem - c1 * PX;
    return ((int64_t)(o[0] + c0) * g.n[1] + (o[1] + c1)) * g.n[2] + (o[2] + c2);
}

// Values every point needs, passed by value; the decompressor's rare outlier
// read goes through shared memory so that no pass keeps it in registers.
struct Hot {
    float eb_f, ebx2_f, r_f;
};

struct Rare {
    const float* out;  // decompress: outlier values were scattered here beforehand
    FieldGeo g;
    int o[3];
};

__shared__ Rare s_rare;

template <int A>
__device__ __noinline__ float outlier_value(int vi)
{
    return s_rare.out[global_index<A>(s_rare.g, s_rare.o, vi)];
}

// compress: quantize x against p, stage the code, return the reconstruction
__device__ __forceinline__ float point_compress(const Hot& h, float xv, float pr, uint8_t* code_slot)
{
    float xr;
    *code_slot = (uint8_t)quantize(xv, pr, h.eb_f, h.ebx2_f, h.r_f, xr);
    return xr;
}

// decompress: the reconstruction from the staged code
template <int A>
__device__ __forceinline__ float point_decompress(const Hot& h, int code, float pr, int vi)
{
    float xr = dequantize(code, pr, h.ebx2_f);
    if (code == 0) xr = outlier_value<A>(vi);
    return xr;
}

// ---------------------------------------------------------------------------
// Passes.  A pass along D predicts, on every line parallel to D, the points
// at odd multiples of S from the nodes at even multiples (stencil cases from
// the extent ED of the line).  Lines are indexed by the two other dims,
// stepping by STQ / STR.
// ---------------------------------------------------------------------------
template <int A, int S, int D, bool CUBIC, bool COMP, bool FULL>
__device__ __forceinline__ void pass_cols(float* __restrict__ v, uint8_t* __restrict__ cs, const Hot h, int stq,
                                          int str, int nq, int nr, int ed)
{
    static_assert(D == 0 || D == 1, "columns");
    using Lw = Lay<A>;
    constexpr int Q = (D == 0) ? 1 : 0;  // the other two dims: Q and 2
    constexpr int NDM = A / (2 * S);
    constexpr int VPD = (D == 0 ? Lw::PY : Lw::PX) * S, VPQ = (Q == 0 ? Lw::PY : Lw::PX);
    constexpr int CX = COMP ? Lw::CXC : Lw::CXD, CY = COMP ? Lw::CYC : Lw::CYD;
    constexpr int CPD = (D == 0 ? CY : CX) * S, CPQ = (Q == 0 ? CY : CX);
    const int nd = FULL ? NDM : ((ed >= S) ? ((ed - S) / (2 * S) + 1) : 0);
    const int nl = nq * nr;
    if constexpr (FULL && NDM >= 4) {
        // whole line: first and last points peeled, the interior loops over
        // the cubic (or linear) midpoint with the nodes sliding through registers
        for (int line = threadIdx.x; line < nl; line += blockDim.x) {
            const int jq = line / nr, jr = line - jq * nr;
            const int cq = jq * stq, cr = jr * str;
            const int vb = cq * VPQ + cr, cb = cq * CPQ + cr;
            float fa = 0.0f, fb = v[vb], fu = v[vb + 2 * VPD], fv = v[vb + 4 * VPD];
            auto point = [&](int k, float pr) {
                const int vi = vb + (2 * k + 1) * VPD;
                if constexpr (COMP)
                    v[vi] = point_compress(h, v[vi], pr, cs + cb + (2 * k + 1) * CPD);
                else
                    v[vi] = point_decompress<A>(h, cs[cb + (2 * k + 1) * CPD], pr, vi);
            };
            point(0, predict(CUBIC, false, true, true, 0.0f, fb, fu, fv));
#pragma unroll 2
            for (int k = 1; k <= NDM - 2; ++k) {
                fa = fb, fb = fu, fu = fv;
                fv = v[vb + (2 * k + 4) * VPD];
                point(k, predict(CUBIC, true, true, true, fa, fb, fu, fv));
            }
            point(NDM - 1, predict(CUBIC, true, true, false, fb, fu, fv, 0.0f));
        }
        return;
    }
    for (int line = threadIdx.x; line < nl; line += blockDim.x) {
        const int jq = line / nr, jr = line - jq * nr;
        const int cq = jq * stq, cr = jr * str;
        const int vb = cq * VPQ + cr, cb = cq * CPQ + cr;
        float f[NDM + 1];  // known nodes at even multiples of S along D
#pragma unroll
        for (int m = 0; m <= NDM; ++m) f[m] = (FULL || 2 * m * S <= ed) ? v[vb + 2 * m * VPD] : 0.0f;
#pragma unroll
        for (int k = 0; k < NDM; ++k) {
            if (!FULL && k >= nd) break;
            const int c = (2 * k + 1) * S;
            const bool have_r = FULL ? true : (c + S <= ed);
            const bool have_r3 = FULL ? (k + 2 <= NDM) : (c + 3 * S <= ed);
            const float pr = predict(CUBIC, k >= 1, have_r, have_r3, k >= 1 ? f[k - 1] : 0.0f, f[k],
                                     have_r ? f[k + 1] : 0.0f, (k + 2 <= NDM && have_r3) ? f[k + 2] : 0.0f);
            const int vi = vb + (2 * k + 1) * VPD;
            if constexpr (COMP) {
                v[vi] = point_compress(h, v[vi], pr, cs + cb + (2 * k + 1) * CPD);
            } else {
                v[vi] = point_decompress<A>(h, cs[cb + (2 * k + 1) * CPD], pr, vi);
            }
        }
    }
}

// Pass along dim 2: one row per thread, moved with 16-byte accesses.
template <int A, int S, bool CUBIC, bool COMP, bool FULL>
__device__ __forceinline__ void pass_rows(float* __restrict__ v, uint8_t* __restrict__ cs, const Hot h, int stq,
                                          int str, int nq, int nr, int ed)
{
    using Lw = Lay<A>;
    constexpr int NDM = A / (2 * S);
    constexpr int NV = A / 4;  // float4 chunks of a row; elements 4*NV .. A one by one
    constexpr int CX = COMP ? Lw::CXC : Lw::CXD, CY = COMP ? Lw::CYC : Lw::CYD;
    constexpr int NCW = (A + 4) / 4;  // code words covering positions 0..A
    const int nd = FULL ? NDM : ((ed >= S) ? ((ed - S) / (2 * S) + 1) : 0);
    const int nl = nq * nr;
    for (int line = threadIdx.x; line < nl; line += blockDim.x) {
        const int jq = line / nr, jr = line - jq * nr;
        const int c0 = jq * stq, c1 = jr * str;
        float* row = v + c0 * Lw::PY + c1 * Lw::PX;
        const int cb = c0 * CY + c1 * CX;
        float r[A + 1];
#pragma unroll
        for (int j = 0; j < NV; ++j) {
            const float4 q = reinterpret_cast<const float4*>(row)[j];
            r[4 * j] = q.x, r[4 * j + 1] = q.y, r[4 * j + 2] = q.z, r[4 * j + 3] = q.w;
        }
#pragma unroll
        for (int j = 4 * NV; j <= A; ++j) r[j] = row[j];
        uint32_t cw[(NCW + 3) / 4 * 4];  // decompress: the row's codes, 4 per word
        if constexpr (!COMP) {
            const uint4* cwp = reinterpret_cast<const uint4*>(cs + cb);
#pragma unroll
            for (int j = 0; j < (NCW + 3) / 4; ++j) {
                const uint4 q = cwp[j];
                cw[4 * j] = q.x, cw[4 * j + 1] = q.y, cw[4 * j + 2] = q.z, cw[4 * j + 3] = q.w;
            }
        }
#pragma unroll
        for (int k = 0; k < NDM; ++k) {
            if (!FULL && k >= nd) break;
            const int c = (2 * k + 1) * S;
            const bool have_r = FULL ? true : (c + S <= ed);
            const bool have_r3 = FULL ? (k + 2 <= NDM) : (c + 3 * S <= ed);
            const float pr = predict(CUBIC, k >= 1, have_r, have_r3, k >= 1 ? r[c - 3 * S] : 0.0f, r[c - S],
                                     have_r ? r[c + S] : 0.0f, (c + 3 * S <= A && have_r3) ? r[c + 3 * S] : 0.0f);
            if constexpr (COMP) {
                r[c] = point_compress(h, r[c], pr, cs + cb + c);
            } else {
                r[c] = point_decompress<A>(h, (cw[c >> 2] >> (8 * (c & 3))) & 0xff, pr,
                                           c0 * Lw::PY + c1 * Lw::PX + c);
            }
        }
#pragma unroll
        for (int j = 0; j < NV; ++j)
            reinterpret_cast<float4*>(row)[j] = make_float4(r[4 * j], r[4 * j + 1], r[4 * j + 2], r[4 * j + 3]);
#pragma unroll
        for (int j = 4 * NV; j < A; ++j) row[j] = r[j];
    }
}

template <int A, int S, int D, bool CUBIC, bool COMP, bool FULL>
__device__ __forceinline__ void pass_any(float* v, uint8_t* cs, const Hot h, int stq, int str, int nq, int nr,
                                         int ed)
{
    if constexpr (D == 2)
        pass_rows<A, S, CUBIC, COMP, FULL>(v, cs, h, stq, str, nq, nr, ed);
    else
        pass_cols<A, S, D, CUBIC, COMP, FULL>(v, cs, h, stq, str, nq, nr, ed);
}

// ---------------------------------------------------------------------------
// Full 3D tiles: the whole level at compile time
// ---------------------------------------------------------------------------
// Step of dim DIM in pass PASS of a level with sequence (D0, D1, D2): dims
// refined earlier in this level step by S, later ones by 2S.
template <int D0, int D1, int D2, int DIM, int PASS, int S>
__host__ __device__ constexpr int step_of()
{
    return ((DIM == D0 ? 0 : (DIM == D1 ? 1 : 2)) < PASS) ? S : 2 * S;
}

template <int A, int S, int D, int PASS, int D0, int D1, int D2, bool CUBIC, bool COMP>
__device__ __forceinline__ void pass_full(float* v, uint8_t* cs, const Hot h)
{
    constexpr int Q = (D == 0) ? 1 : 0, R = (D == 2) ? 1 : 2;
    constexpr int STQ = step_of<D0, D1, D2, Q, PASS, S>(), STR = step_of<D0, D1, D2, R, PASS, S>();
    pass_any<A, S, D, CUBIC, COMP, true>(v, cs, h, STQ, STR, A / STQ + 1, A / STR + 1, A);
}

template <int A, int S, int D0, int D1, int D2, bool CUBIC, bool COMP>
__device__ __noinline__ void level_full(float* v, uint8_t* cs, const Hot h)
{
    pass_full<A, S, D0, 0, D0, D1, D2, CUBIC, COMP>(v, cs, h);
    __syncthreads();
    pass_full<A, S, D1, 1, D0, D1, D2, CUBIC, COMP>(v, cs, h);
    __syncthreads();
    pass_full<A, S, D2, 2, D0, D1, D2, CUBIC, COMP>(v, cs, h);
    __syncthreads();
}

// sel = 2 * perm + cubic; perm: 0 (0,1,2) 1 (0,2,1) 2 (1,0,2) 3 (1,2,0) 4 (2,0,1) 5 (2,1,0)
template <int A, int S, bool COMP>
__device__ __forceinline__ void level_dispatch(int sel, float* v, uint8_t* cs, const Hot h)
{
    switch (sel) {
    case 0: level_full<A, S, 0, 1, 2, false, COMP>(v, cs, h); break;
    case 1: level_full<A, S, 0, 1, 2, true, COMP>(v, cs, h); break;
    case 2: level_full<A, S, 0, 2, 1, false, COMP>(v, cs, h); break;
    case 3: level_full<A, S, 0, 2, 1, true, COMP>(v, cs, h); break;
    case 4: level_full<A, S, 1, 0, 2, false, COMP>(v, cs, h); break;
    case 5: level_full<A, S, 1, 0, 2, true, COMP>(v, cs, h); break;
    case 6: level_full<A, S, 1, 2, 0, false, COMP>(v, cs, h); break;
    case 7: level_full<A, S, 1, 2, 0, true, COMP>(v, cs, h); break;
    case 8: level_full<A, S, 2, 0, 1, false, COMP>(v, cs, h); break;
    case 9: level_full<A, S, 2, 0, 1, true, COMP>(v, cs, h); break;
    case 10: level_full<A, S, 2, 1, 0, false, COMP>(v, cs, h); break;
    default: level_full<A, S, 2, 1, 0, true, COMP>(v, cs, h); break;
    }
}

template <int A, int LV, bool COMP>
__device__ __forceinline__ void levels_full(const int* s_sel, float* v, uint8_t* cs, const Hot h)
{
    level_dispatch<A, (1 << LV), COMP>(s_sel[LV], v, cs, h);
    if constexpr (LV > 0) levels_full<A, LV - 1, COMP>(s_sel, v, cs, h);
}

__device__ __forceinline__ int perm_sel(const hi_level& lv)
{
    const int a = lv.order[0], b = lv.order[1];
    const int p = (a == 0) ? (b == 1 ? 0 : 1) : (a == 1) ? (b == 0 ? 2 : 3) : (b == 0 ? 4 : 5);
    return 2 * p + (lv.interp == HI_CUBIC ? 1 : 0);
}

template <int A>
struct HasFull {
    static constexpr bool value = (A == 8 || A == 16);
};

// ---------------------------------------------------------------------------
// Other tiles: extents at run time, one instantiation per (level, dim, spline)
// ---------------------------------------------------------------------------
__device__ __forceinline__ int pick3(const int a[3], int i) { return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]); }

template <int A, int S, int D, bool COMP>
__device__ __forceinline__ void pass_dispatch(bool cubic, float* v, uint8_t* cs, const Hot h, int stq, int str,
                                              int nq, int nr, int ed)
{
    if (ed == A) {  // the pass dim is whole: only the line counts are shorter
        if (cubic)
            pass_any<A, S, D, true, COMP, true>(v, cs, h, stq, str, nq, nr, ed);
        else
            pass_any<A, S, D, false, COMP, true>(v, cs, h, stq, str, nq, nr, ed);
    } else {
        if (cubic)
            pass_any<A, S, D, true, COMP, false>(v, cs, h, stq, str, nq, nr, ed);
        else
            pass_any<A, S, D, false, COMP, false>(v, cs, h, stq, str, nq, nr, ed);
    }
}

template <int A, int LV, bool COMP>
__device__ __noinline__ void level_ragged(const hi_level lv, float* v, uint8_t* cs, const Hot h, int e0, int e1,
                                          int e2)
{
    constexpr int S = 1 << LV;
    const bool cubic = lv.interp == HI_CUBIC;
    const int e[3] = {e0, e1, e2};
    for (int p = 0; p < 3; ++p) {
        const int d = lv.order[p];
        const int q = (d == 0) ? 1 : 0, r = (d == 2) ? 1 : 2;
        const int posq = (lv.order[0] == q) ? 0 : ((lv.order[1] == q) ? 1 : 2);
        const int posr = (lv.order[0] == r) ? 0 : ((lv.order[1] == r) ? 1 : 2);
        const int stq = (posq < p) ? S : 2 * S, str = (posr < p) ? S : 2 * S;
        const int ed = pick3(e, d);
        if (ed < S) continue;  // no point on this pass (CTA-uniform)
        const int nq = pick3(e, q) / stq + 1, nr = pick3(e, r) / str + 1;
        if (d == 0)
            pass_dispatch<A, S, 0, COMP>(cubic, v, cs, h, stq, str, nq, nr, ed);
        else if (d == 1)
            pass_dispatch<A, S, 1, COMP>(cubic, v, cs, h, stq, str, nq, nr, ed);
        else
            pass_dispatch<A, S, 2, COMP>(cubic, v, cs, h, stq, str, nq, nr, ed);
        __syncthreads();
    }
}

template <int A, int LV, bool COMP>
__device__ __forceinline__ void levels_ragged(const hi_level* s_lv, float* v, uint8_t* cs, const Hot h,
                                              const TileInfo& ti)
{
    level_ragged<A, LV, COMP>(s_lv[LV], v, cs, h, ti.e[0], ti.e[1], ti.e[2]);
    if constexpr (LV > 0) levels_ragged<A, LV - 1, COMP>(s_lv, v, cs, h, ti);
}

// ---------------------------------------------------------------------------
// Staging
// ---------------------------------------------------------------------------
template <int A>
__device__ void load_tile_plain(float* v, const float* __restrict__ x, const FieldGeo& g, const TileInfo& ti)
{
    using Lw = Lay<A>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rows = (ti.e[0] + 1) * (ti.e[1] + 1);
    for (int rr = warp; rr < rows; rr += nw) {
        const int c0 = rr / (ti.e[1] + 1);
        const int c1 = rr - c0 * (ti.e[1] + 1);
        const float* src = x + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2];
        for (int c2 = lane; c2 <= ti.e[2]; c2 += 32) v[c0 * Lw::PY + c1 * Lw::PX + c2] = src[c2];
    }
}

template <int A>
__device__ void load_codes_plain(uint8_t* cs, const uint8_t* __restrict__ codes, const FieldGeo& g,
                                 const TileInfo& ti)
{
    using Lw = Lay<A>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rows = (ti.e[0] + 1) * (ti.e[1] + 1);
    for (int rr = warp; rr < rows; rr += nw) {
        const int c0 = rr / (ti.e[1] + 1);
        const int c1 = rr - c0 * (ti.e[1] + 1);
        const uint8_t* src = codes + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2];
        for (int c2 = lane; c2 <= ti.e[2]; c2 += 32) cs[c0 * Lw::CYD + c1 * Lw::CXD + c2] = src[c2];
    }
}

__device__ __forceinline__ void tma_issue(void* dst, const CUtensorMap* map, const FieldGeo& g, int tile, int A,
                                          uint64_t* mbar, uint32_t bytes)
{
    int t[3];
    tile_coords(g, tile, t);
    mbar_arrive_expect_tx(mbar, bytes);
    tma_load_3d(dst, map, t[2] * A, t[1] * A, t[0] * A, mbar);
}

// ---------------------------------------------------------------------------
// Epilogue helpers (all lanes of the warp call them)
// ---------------------------------------------------------------------------
// Outliers (code 0) of the tile, one candidate per lane: the warp reserves
// its slots in the output list with one atomic and writes them.
template <int A>
__device__ __forceinline__ void outlier_append(bool is_out, int vi, const float* v, hi_header* hdr,
                                               uint32_t* out_idx, float* out_val, uint64_t out_cap,
                                               const FieldGeo& g, const int o[3])
{
    const unsigned m = __ballot_sync(0xffffffffu, is_out);
    if (m == 0) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader)
        base = atomicAdd(reinterpret_cast<unsigned long long*>(&hdr->n_outliers), (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (!is_out) return;
    const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
    if (pos < out_cap) {
        out_idx[pos] = (uint32_t)global_index<A>(g, o, vi);
        out_val[pos] = v[vi];
    } else {
        set_status(&hdr->status, HI_ECAPACITY);
    }
}

// Histogram: codes 120..135 (the bulk at any practical error bound) go to
// per-thread 16-bit counters laid out bin-major, so that a warp's updates hit
// 32 consecutive half-words (no bank conflict, no atomics); other codes go
// to shared-memory atomics.  Folded into the CTA histogram at kernel end.
constexpr int kHistLo = 120, kHistBins = 16;

__device__ __forceinline__ void hist_count(uint16_t* hc, uint32_t* s_hist, int code, bool valid)
{
    const unsigned k = (unsigned)(code - kHistLo);
    if (valid) {
        if (k < (unsigned)kHistBins)
            hc[k * blockDim.x + threadIdx.x] += 1;
        else
            atomicAdd(&s_hist[code], 1u);
    }
}

// ---------------------------------------------------------------------------
// Predict + quantize
// ---------------------------------------------------------------------------
template <int A>
__global__ void __launch_bounds__(kMaxThreads, 4)
    k_compress(const __grid_constant__ CUtensorMap tmap, const FieldGeo g, const float* __restrict__ x,
               uint8_t* __restrict__ codes, float* __restrict__ anchors, uint32_t* __restrict__ out_idx,
               float* __restrict__ out_val, const uint64_t out_cap, uint32_t* __restrict__ hist_g,
               float* __restrict__ recon_g, hi_header* __restrict__ hdr, uint32_t* __restrict__ queue,
               const uint32_t tma_bytes, const int flags)
{
    using Lw = Lay<A>;
    extern __shared__ __align__(128) unsigned char smem[];
    const bool dbuf = flags & kFlagDoubleBuf;
    const int vb_bytes = vbuf_bytes<A>(g.b0);
    float* vbuf[2] = {reinterpret_cast<float*>(smem), reinterpret_cast<float*>(smem + (dbuf ? vb_bytes : 0))};
    uint8_t* cs = smem + (dbuf ? 2 : 1) * vb_bytes;
    uint16_t* hc = reinterpret_cast<uint16_t*>(cs + round128(g.b0 * Lw::P * Lw::CXC));  // [kHistBins][threads]
    __shared__ uint32_t s_hist[256];
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ hi_level s_lv[HI_MAX_LEVELS];
    __shared__ int s_sel[HI_MAX_LEVELS];
    __shared__ int s_next;
    __shared__ TileInfo s_ti[2];  // this tile's geometry and the next one's (thread 0 decodes)

    const int tid = threadIdx.x;
    const bool use_tma = flags & kFlagTma;
    {   // an earlier stage failed (bad range, device-side EINVAL): leave outputs untouched
        const uint32_t st = hdr->status;
        if (__syncthreads_or(st != 0 && st != HI_ECAPACITY)) return;
    }
    Hot h;
    h.eb_f = hdr->eb_f;
    h.ebx2_f = hdr->ebx2_f;
    h.r_f = hdr->r_f;
    const bool hist_on = hist_g != nullptr;

    for (int i = tid; i < 256; i += blockDim.x) s_hist[i] = 0;
    if (hist_on)
        for (int k = 0; k < kHistBins; ++k) hc[k * blockDim.x + tid] = 0;
    if (tid < HI_MAX_LEVELS) {
        s_lv[tid] = hdr->level[tid];
        s_sel[tid] = perm_sel(s_lv[tid]);
    }
    if (tid == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        fence_mbar_init();
        if ((int)blockIdx.x < g.ntiles) s_ti[0] = tile_info<A>(g, blockIdx.x);
        if (use_tma) {
            prefetch_tmap(&tmap);
            if ((int)blockIdx.x < g.ntiles) tma_issue(vbuf[0], &tmap, g, blockIdx.x, A, &s_mbar[0], tma_bytes);
        }
    }
    __syncthreads();
    const bool full_ok = HasFull<A>::value && g.n[0] > 1 && g.n[1] > 1 && g.n[2] > 1;

    // tiles after each CTA's first come from a queue in ascending order: the
    // load stays balanced (edge tiles cost more) and neighbouring tiles, which
    // share faces, are in flight together
    int it = 0;
    for (int tile = blockIdx.x; tile < g.ntiles; ++it) {
        const int buf = dbuf ? (it & 1) : 0;
        float* v = vbuf[buf];
        const TileInfo ti = s_ti[it & 1];
        if (tid == 0) {
            const int nx = (int)gridDim.x + (int)atomicAdd(queue, 1u);
            s_next = nx;
            if (nx < g.ntiles) s_ti[(it + 1) & 1] = tile_info<A>(g, nx);
            if (use_tma && dbuf && nx < g.ntiles)
                tma_issue(vbuf[buf ^ 1], &tmap, g, nx, A, &s_mbar[buf ^ 1], tma_bytes);
            if (use_tma && !dbuf && it > 0) tma_issue(v, &tmap, g, tile, A, &s_mbar[0], tma_bytes);
        }
        if (tid < 8) {  // anchors keep the zero-error code
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            if (a0 * A <= ti.e[0] && a1 * A <= ti.e[1] && a2 * A <= ti.e[2])
                cs[a0 * A * Lw::CYC + a1 * A * Lw::CXC + a2 * A] = (uint8_t)kRadius;
        }
        if (use_tma) {
            const bool ok = mbar_wait(&s_mbar[buf], dbuf ? ((it >> 1) & 1) : (it & 1), kSpinLimit);
            if (!__syncthreads_and(ok)) {
                if (tid == 0) set_status(&hdr->status, HI_ETIMEOUT);
                if (dbuf && s_next < g.ntiles) mbar_wait(&s_mbar[buf ^ 1], ((it + 1) >> 1) & 1, kSpinLimit);
                return;
            }
        } else {
            load_tile_plain<A>(v, x, g, ti);
            __syncthreads();
        }
        const int next = s_next;
        const bool full = full_ok && ti.e[0] == A && ti.e[1] == A && ti.e[2] == A;
        if constexpr (HasFull<A>::value) {
            if (full)
                levels_full<A, TileGeom<A>::L - 1, true>(s_sel, v, cs, h);
            else
                levels_ragged<A, TileGeom<A>::L - 1, true>(s_lv, v, cs, h, ti);
        } else {
            levels_ragged<A, TileGeom<A>::L - 1, true>(s_lv, v, cs, h, ti);
        }

        // ---- epilogue: owned codes, histogram and outliers; recon; anchors
        const int own0 = ti.own[0] + 1, own1 = ti.own[1] + 1, own2 = ti.own[2] + 1;
        const int rows = own0 * own1;
        const bool vec_codes = (flags & kFlagVecCodes) && own2 == A && A >= 8;
        if (vec_codes) {
            constexpr int CH = (A >= 16) ? 4 : 2;  // words per global vector store
            constexpr int NCH = (A >= 8) ? A / (4 * CH) : 1;
            const bool square = own0 == A && own1 == A;  // rows decompose with shifts
            const int items = rows * NCH;
            for (int i0 = 0; i0 < items; i0 += blockDim.x) {
                const int i = i0 + tid;
                const bool act = i < items;
                const int row = act ? i / NCH : 0, ch = act ? i - row * NCH : 0;
                const int c0 = square ? row / A : row / own1;
                const int c1 = row - c0 * (square ? A : own1);
                const uint32_t* src = reinterpret_cast<const uint32_t*>(cs + c0 * Lw::CYC + c1 * Lw::CXC) + ch * CH;
                uint8_t* dst = codes + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] +
                               ch * CH * 4;
                uint32_t w[4];
                uint32_t z = 0;  // nonzero iff some code of the chunk is 0 (an outlier)
#pragma unroll
                for (int j = 0; j < CH; ++j) {
                    w[j] = src[j];
                    z |= (w[j] - 0x01010101u) & ~w[j] & 0x80808080u;
                }
                if (act) {
                    if constexpr (CH == 4)
                        *reinterpret_cast<uint4*>(dst) = make_uint4(w[0], w[1], w[2], w[3]);
                    else
                        *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
                }
                if (__any_sync(0xffffffffu, act && z != 0)) {
#pragma unroll
                    for (int b = 0; b < 4 * CH; ++b) {
                        const int code = (w[b >> 2] >> (8 * (b & 3))) & 0xff;
                        outlier_append<A>(act && code == 0, c0 * Lw::PY + c1 * Lw::PX + ch * CH * 4 + b, v, hdr,
                                          out_idx, out_val, out_cap, g, ti.o);
                    }
                }
                if (hist_on) {
#pragma unroll
                    for (int b = 0; b < 4 * CH; ++b) hist_count(hc, s_hist, (w[b >> 2] >> (8 * (b & 3))) & 0xff, act);
                }
            }
        } else {
            const int items = rows * own2;
            for (int i0 = 0; i0 < items; i0 += blockDim.x) {
                const int i = i0 + tid;
                const bool act = i < items;
                const int row = act ? i / own2 : 0, c2 = act ? i - row * own2 : 0;
                const int c0 = row / own1, c1 = row - c0 * own1;
                const int code = cs[c0 * Lw::CYC + c1 * Lw::CXC + c2];
                if (act)
                    codes[((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2] =
                        (uint8_t)code;
                if (hist_on) hist_count(hc, s_hist, code, act);
                outlier_append<A>(act && code == 0, c0 * Lw::PY + c1 * Lw::PX + c2, v, hdr, out_idx, out_val, out_cap,
                                  g, ti.o);
            }
        }
        if (recon_g) {
            const int items = rows * own2;
            for (int i = tid; i < items; i += blockDim.x) {
                const int row = i / own2, c2 = i - row * own2;
                const int c0 = row / own1, c1 = row - c0 * own1;
                recon_g[((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2] =
                    v[c0 * Lw::PY + c1 * Lw::PX + c2];
            }
        }
        if (tid < 8) {  // owned anchors, verbatim (Sec. 3.2)
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            const int l0 = a0 * A, l1 = a1 * A, l2 = a2 * A;
            if (l0 <= ti.own[0] && l1 <= ti.own[1] && l2 <= ti.own[2]) {
                const int64_t ai = ((int64_t)(ti.o[0] / A + a0) * g.na[1] + (ti.o[1] / A + a1)) * g.na[2] +
                                   (ti.o[2] / A + a2);
                anchors[ai] = v[l0 * Lw::PY + l1 * Lw::PX + l2];
                if (hist_on) atomicSub(&s_hist[kRadius], 1u);  // anchors are not predicted
            }
        }
        // keep the buffers until every thread is done; order the generic-proxy
        // writes above before the TMA overwrite of this buffer
        fence_proxy_async_smem();
        __syncthreads();
        tile = next;
    }
    if (hist_on) {
        for (int k = 0; k < kHistBins; ++k) {  // fold this thread's counters, a warp at a time
            uint32_t c = hc[k * blockDim.x + tid];
            for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
            if ((tid & 31) == 0) atomicAdd(&s_hist[kHistLo + k], c);
        }
        __syncthreads();
        for (int i = tid; i < 256; i += blockDim.x)
            if (s_hist[i]) atomicAdd(&hist_g[i], s_hist[i]);
    }
}

// ---------------------------------------------------------------------------
// Reconstruct
// ---------------------------------------------------------------------------
template <int A>
__global__ void __launch_bounds__(kMaxThreads, 4)
    k_decompress(const __grid_constant__ CUtensorMap cmap, const FieldGeo g, const uint8_t* __restrict__ codes,
                 const float* __restrict__ anchors, float* out, const hi_header* __restrict__ hdr,
                 uint32_t* __restrict__ status, uint32_t* __restrict__ queue, const uint32_t tma_bytes,
                 const int flags)
{
    using Lw = Lay<A>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int vb_bytes = vbuf_bytes<A>(g.b0);
    const int cb_bytes = round128(g.b0 * Lw::P * Lw::CXD);
    const bool dbuf = flags & kFlagDoubleBuf;
    float* v = reinterpret_cast<float*>(smem);
    uint8_t* cbuf[2] = {smem + vb_bytes, smem + vb_bytes + (dbuf ? cb_bytes : 0)};
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ hi_level s_lv[HI_MAX_LEVELS];
    __shared__ int s_sel[HI_MAX_LEVELS];
    __shared__ int s_next;
    __shared__ TileInfo s_ti[2];

    const int tid = threadIdx.x;
    const bool use_tma = flags & kFlagTma;
    if (__syncthreads_or(status != nullptr && *status != 0)) return;
    Hot h;
    h.eb_f = 0.0f;
    h.ebx2_f = hdr->ebx2_f;
    h.r_f = 0.0f;
    if (tid == 0) {
        s_rare.out = out;
        s_rare.g = g;
    }
    if (tid < HI_MAX_LEVELS) {
        s_lv[tid] = hdr->level[tid];
        s_sel[tid] = perm_sel(s_lv[tid]);
    }
    if (tid == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        fence_mbar_init();
        if ((int)blockIdx.x < g.ntiles) s_ti[0] = tile_info<A>(g, blockIdx.x);
        if (use_tma) {
            prefetch_tmap(&cmap);
            if ((int)blockIdx.x < g.ntiles) tma_issue(cbuf[0], &cmap, g, blockIdx.x, A, &s_mbar[0], tma_bytes);
        }
    }
    __syncthreads();
    const bool full_ok = HasFull<A>::value && g.n[0] > 1 && g.n[1] > 1 && g.n[2] > 1;

    // the 8 corner anchors of a tile, loaded one tile ahead by threads 0..7
    auto anchor_of = [&](int pos, const TileInfo& tn) -> float {
        if (tid >= 8 || pos >= g.ntiles) return 0.0f;
        const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
        if (a0 * A > tn.e[0] || a1 * A > tn.e[1] || a2 * A > tn.e[2]) return 0.0f;
        return anchors[((int64_t)(tn.o[0] / A + a0) * g.na[1] + (tn.o[1] / A + a1)) * g.na[2] + (tn.o[2] / A + a2)];
    };
    float a_cur = anchor_of(blockIdx.x, s_ti[0]);

    int it = 0;
    for (int tile = blockIdx.x; tile < g.ntiles; ++it) {
        const int buf = dbuf ? (it & 1) : 0;
        uint8_t* cs = cbuf[buf];
        const TileInfo ti = s_ti[it & 1];
        if (tid == 0) {
            const int nx = (int)gridDim.x + (int)atomicAdd(queue, 1u);
            s_next = nx;
            if (nx < g.ntiles) s_ti[(it + 1) & 1] = tile_info<A>(g, nx);
            s_rare.o[0] = ti.o[0], s_rare.o[1] = ti.o[1], s_rare.o[2] = ti.o[2];
            if (use_tma && dbuf && nx < g.ntiles)
                tma_issue(cbuf[buf ^ 1], &cmap, g, nx, A, &s_mbar[buf ^ 1], tma_bytes);
            if (use_tma && !dbuf && it > 0) tma_issue(cs, &cmap, g, tile, A, &s_mbar[0], tma_bytes);
        }
        if (tid < 8) {  // seed the anchors
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            const int l0 = a0 * A, l1 = a1 * A, l2 = a2 * A;
            if (l0 <= ti.e[0] && l1 <= ti.e[1] && l2 <= ti.e[2]) v[l0 * Lw::PY + l1 * Lw::PX + l2] = a_cur;
        }
        if (use_tma) {
            const bool ok = mbar_wait(&s_mbar[buf], dbuf ? ((it >> 1) & 1) : (it & 1), kSpinLimit);
            if (!__syncthreads_and(ok)) {
                if (tid == 0) set_status(status, HI_ETIMEOUT);
                if (dbuf && s_next < g.ntiles) mbar_wait(&s_mbar[buf ^ 1], ((it + 1) >> 1) & 1, kSpinLimit);
                return;
            }
        } else {
            load_codes_plain<A>(cs, codes, g, ti);
            __syncthreads();
        }
        const int next = s_next;
        const float a_nxt = anchor_of(next, s_ti[(it + 1) & 1]);  // in flight while this tile is reconstructed
        const bool full = full_ok && ti.e[0] == A && ti.e[1] == A && ti.e[2] == A;
        if constexpr (HasFull<A>::value) {
            if (full)
                levels_full<A, TileGeom<A>::L - 1, false>(s_sel, v, cs, h);
            else
                levels_ragged<A, TileGeom<A>::L - 1, false>(s_lv, v, cs, h, ti);
        } else {
            levels_ragged<A, TileGeom<A>::L - 1, false>(s_lv, v, cs, h, ti);
        }

        // ---- epilogue: owned reconstructed values
        const int own0 = ti.own[0] + 1, own1 = ti.own[1] + 1, own2 = ti.own[2] + 1;
        const int rows = own0 * own1;
        const bool vec_out = (flags & kFlagVecOut) && own2 == A && A >= 4;
        if (vec_out) {
            constexpr int NCH = (A >= 4) ? A / 4 : 1;
            const bool square = own0 == A && own1 == A;  // rows decompose with shifts
            const int items = rows * NCH;
            for (int i = tid; i < items; i += blockDim.x) {
                const int row = i / NCH, ch = i - row * NCH;
                const int c0 = square ? row / A : row / own1;
                const int c1 = row - c0 * (square ? A : own1);
                const float4 f4 = *reinterpret_cast<const float4*>(v + c0 * Lw::PY + c1 * Lw::PX + ch * 4);
                *reinterpret_cast<float4*>(out + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] +
                                           ti.o[2] + ch * 4) = f4;
            }
        } else {
            const int items = rows * own2;
            for (int i = tid; i < items; i += blockDim.x) {
                const int row = i / own2, c2 = i - row * own2;
                const int c0 = row / own1, c1 = row - c0 * own1;
                out[((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2] =
                    v[c0 * Lw::PY + c1 * Lw::PX + c2];
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
        tile = next;
        a_cur = a_nxt;
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int A>
size_t compress_smem_t(int b0, bool dbuf, int threads)
{
    return (dbuf ? 2 : 1) * (size_t)vbuf_bytes<A>(b0) + (size_t)round128(b0 * Lay<A>::P * Lay<A>::CXC) +
           (size_t)kHistBins * threads * sizeof(uint16_t);
}

template <int A>
size_t decompress_smem_t(int b0, bool dbuf)
{
    return (size_t)vbuf_bytes<A>(b0) + (dbuf ? 2 : 1) * (size_t)round128(b0 * Lay<A>::P * Lay<A>::CXD);
}

// Double buffering when both buffers and the kernel's static shared memory fit.
template <typename K>
static bool fits_double(K kern, size_t dyn_double)
{
    int dev = 0, optin = 0;
    cudaFuncAttributes fa;
    if (cudaGetDevice(&dev) != cudaSuccess) return false;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return false;
    if (cudaFuncGetAttributes(&fa, kern) != cudaSuccess) return false;
    return dyn_double + fa.sharedSizeBytes <= (size_t)optin;
}

template <typename K>
static cudaError_t persistent_grid(K kern, int threads, size_t smem, int num_sms, int ntiles, int max_ctas, int* grid)
{
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    int g = per_sm * num_sms;
    if (g > ntiles) g = ntiles;
    if (max_ctas > 0 && g > max_ctas) g = max_ctas;
    *grid = g > 0 ? g : 1;
    return cudaSuccess;
}

template <int A>
static cudaError_t launch_compress_t(const CompressLaunch& c, cudaStream_t st)
{
    auto kern = k_compress<A>;
    const bool dbuf = c.buffers == 2 && fits_double(kern, compress_smem_t<A>(c.g.b0, true, c.threads));
    const size_t smem = compress_smem_t<A>(c.g.b0, dbuf, c.threads);
    int grid = 0;
    cudaError_t err = persistent_grid(kern, c.threads, smem, c.num_sms, c.g.ntiles, c.max_ctas, &grid);
    if (err != cudaSuccess) return err;
    kern<<<grid, c.threads, smem, st>>>(c.tmap, c.g, c.x, c.codes, c.anchors, c.out_idx, c.out_val, c.out_cap,
                                        c.hist, c.recon, c.hdr, c.queue, c.tma_bytes,
                                        c.flags | (dbuf ? kFlagDoubleBuf : 0));
    return cudaGetLastError();
}

template <int A>
static cudaError_t launch_decompress_t(const DecompressLaunch& c, cudaStream_t st)
{
    auto kern = k_decompress<A>;
    const bool dbuf = c.buffers == 2 && fits_double(kern, decompress_smem_t<A>(c.g.b0, true));
    const size_t smem = decompress_smem_t<A>(c.g.b0, dbuf);
    int grid = 0;
    cudaError_t err = persistent_grid(kern, c.threads, smem, c.num_sms, c.g.ntiles, c.max_ctas, &grid);
    if (err != cudaSuccess) return err;
    kern<<<grid, c.threads, smem, st>>>(c.cmap, c.g, c.codes, c.anchors, c.out, c.hdr, c.status, c.queue,
                                        c.tma_bytes, c.flags | (dbuf ? kFlagDoubleBuf : 0));
    return cudaGetLastError();
}

cudaError_t launch_compress(int A, const CompressLaunch& c, cudaStream_t st)
{
    switch (A) {
    case 2: return launch_compress_t<2>(c, st);
    case 4: return launch_compress_t<4>(c, st);
    case 8: return launch_compress_t<8>(c, st);
    case 16: return launch_compress_t<16>(c, st);
    case 32: return launch_compress_t<32>(c, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_decompress(int A, const DecompressLaunch& c, cudaStream_t st)
{
    switch (A) {
    case 2: return launch_decompress_t<2>(c, st);
    case 4: return launch_decompress_t<4>(c, st);
    case 8: return launch_decompress_t<8>(c, st);
    case 16: return launch_decompress_t<16>(c, st);
    case 32: return launch_decompress_t<32>(c, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t compress_smem_bytes(int A, int b0)
{
    switch (A) {
    case 2: return compress_smem_t<2>(b0, false, 256);
    case 4: return compress_smem_t<4>(b0, false, 256);
    case 8: return compress_smem_t<8>(b0, false, 256);
    case 16: return compress_smem_t<16>(b0, false, 256);
    case 32: return compress_smem_t<32>(b0, false, 256);
    default: return 0;
    }
}

}  // namespace hi
