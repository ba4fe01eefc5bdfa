// hi_passes.cuh -- the tile machinery shared by the fused interpolation-predict
// + quantize kernel and its inverse, the level-by-level reconstruction (cuSZ-Hi, arXiv 2507.11165,
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
//     extents at run time (one instantiation per level, dim and spline).
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
#pragma once
#include <cstdint>
#include <map>
#include <mutex>

#include "hi_device.cuh"
#include "hi_internal.h"

// Level functions are inlined into the compress kernel; the reconstruct
// kernel keeps them as calls, which leaves it more registers per pass.
#ifndef HI_LEVEL_FN
#define HI_LEVEL_FN __forceinline__
#endif

namespace hi {

constexpr int kMaxThreads = 128;  // CTA size cap: one 17^3 tile per CTA keeps 128 threads busy

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
// One point of a column pass: float offset vi, code offset ci, prediction pr.
template <int A, bool COMP>
__device__ __forceinline__ void line_point(float* __restrict__ v, uint8_t* __restrict__ cs, const Hot& h, int vi,
                                           int ci, float pr)
{
    if constexpr (COMP)
        v[vi] = point_compress(h, v[vi], pr, cs + ci);
    else
        v[vi] = point_decompress<A>(h, cs[ci], pr, vi);
}

// Line index -> (jq, jr) for nr lines along R.  With run-time line counts the
// quotient comes from a float reciprocal: for line < 2^16 and nr <= 64 the
// product is within 1e-3 of the exact quotient, whose fractional part stays
// at least 1/(2 nr) away from an integer, so the truncation is exact.
template <bool RT>
__device__ __forceinline__ int line_q(int line, int nr, float inv_nr)
{
    if constexpr (RT)
        return (int)__fmul_rn(__fadd_rn((float)line, 0.5f), inv_nr);
    else
        return line / nr;
}

// ED: the pass dim's extent when known at compile time (A for a whole tile),
// 0 when it is only known at run time (the other tiles).
template <int A, int S, int D, bool CUBIC, bool COMP, int ED, bool RT>
__device__ __forceinline__ void pass_cols(float* __restrict__ v, uint8_t* __restrict__ cs, const Hot h, int stq,
                                          int str, int nq, int nr, int ed_rt)
{
    static_assert(D == 0 || D == 1, "columns");
    using Lw = Lay<A>;
    constexpr int Q = (D == 0) ? 1 : 0;  // the other two dims: Q and 2
    constexpr int NDM = A / (2 * S);
    constexpr int VPD = (D == 0 ? Lw::PY : Lw::PX) * S, VPQ = (Q == 0 ? Lw::PY : Lw::PX);
    constexpr int CX = COMP ? Lw::CXC : Lw::CXD, CY = COMP ? Lw::CYC : Lw::CYD;
    constexpr int CPD = (D == 0 ? CY : CX) * S, CPQ = (Q == 0 ? CY : CX);
    const int ed = ED ? ED : ed_rt;
    const int nd = (ed >= S) ? ((ed - S) / (2 * S) + 1) : 0;
    const int nl = nq * nr;
    const float inv_nr = RT ? __frcp_rn((float)nr) : 0.0f;
    if constexpr (ED == A && NDM >= 4) {
        // whole line: first and last points peeled, the interior loops over
        // the cubic (or linear) midpoint with the nodes sliding through registers
        for (int line = threadIdx.x; line < nl; line += blockDim.x) {
            const int jq = line_q<RT>(line, nr, inv_nr), jr = line - jq * nr;
            const int cq = jq * stq, cr = jr * str;
            const int vb = cq * VPQ + cr, cb = cq * CPQ + cr;
            float fa = 0.0f, fb = v[vb], fu = v[vb + 2 * VPD], fv = v[vb + 4 * VPD];
            line_point<A, COMP>(v, cs, h, vb + VPD, cb + CPD, predict(CUBIC, false, true, true, 0.0f, fb, fu, fv));
#pragma unroll
            for (int k = 1; k <= NDM - 2; ++k) {
                fa = fb, fb = fu, fu = fv;
                fv = v[vb + (2 * k + 4) * VPD];
                line_point<A, COMP>(v, cs, h, vb + (2 * k + 1) * VPD, cb + (2 * k + 1) * CPD,
                                    predict(CUBIC, true, true, true, fa, fb, fu, fv));
            }
            line_point<A, COMP>(v, cs, h, vb + (2 * NDM - 1) * VPD, cb + (2 * NDM - 1) * CPD,
                                predict(CUBIC, true, true, false, fb, fu, fv, 0.0f));
        }
    } else {
        for (int line = threadIdx.x; line < nl; line += blockDim.x) {
            const int jq = line_q<RT>(line, nr, inv_nr), jr = line - jq * nr;
            const int cq = jq * stq, cr = jr * str;
            const int vb = cq * VPQ + cr, cb = cq * CPQ + cr;
            float f[NDM + 1];  // known nodes at even multiples of S along D
#pragma unroll
            for (int m = 0; m <= NDM; ++m) f[m] = (2 * m * S <= ed) ? v[vb + 2 * m * VPD] : 0.0f;
#pragma unroll
            for (int k = 0; k < NDM; ++k) {
                if (k >= nd) break;
                const int c = (2 * k + 1) * S;
                const bool have_r = c + S <= ed;
                const bool have_r3 = c + 3 * S <= ed;
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
}

// Pass along dim 2: one row per thread, moved with 16-byte accesses.
template <int A, int S, bool CUBIC, bool COMP, int ED, bool RT>
__device__ __forceinline__ void pass_rows(float* __restrict__ v, uint8_t* __restrict__ cs, const Hot h, int stq,
                                          int str, int nq, int nr, int ed_rt)
{
    using Lw = Lay<A>;
    constexpr int NDM = A / (2 * S);
    constexpr int NV = A / 4;  // float4 chunks of a row; elements 4*NV .. A one by one
    constexpr int CX = COMP ? Lw::CXC : Lw::CXD, CY = COMP ? Lw::CYC : Lw::CYD;
    constexpr int NCW = (A + 4) / 4;  // code words covering positions 0..A
    const int ed = ED ? ED : ed_rt;
    const int nd = (ed >= S) ? ((ed - S) / (2 * S) + 1) : 0;
    const int nl = nq * nr;
    const float inv_nr = RT ? __frcp_rn((float)nr) : 0.0f;
    for (int line = threadIdx.x; line < nl; line += blockDim.x) {
        const int jq = line_q<RT>(line, nr, inv_nr), jr = line - jq * nr;
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
            if (k >= nd) break;
            const int c = (2 * k + 1) * S;
            const bool have_r = c + S <= ed;
            const bool have_r3 = c + 3 * S <= ed;
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

template <int A, int S, int D, bool CUBIC, bool COMP, int ED, bool RT>
__device__ __forceinline__ void pass_any(float* v, uint8_t* cs, const Hot h, int stq, int str, int nq, int nr,
                                         int ed)
{
    if constexpr (D == 2)
        pass_rows<A, S, CUBIC, COMP, ED, RT>(v, cs, h, stq, str, nq, nr, ed);
    else
        pass_cols<A, S, D, CUBIC, COMP, ED, RT>(v, cs, h, stq, str, nq, nr, ed);
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
    pass_any<A, S, D, CUBIC, COMP, A, false>(v, cs, h, STQ, STR, A / STQ + 1, A / STR + 1, A);
}

template <int A, int S, int D0, int D1, int D2, bool CUBIC, bool COMP>
__device__ HI_LEVEL_FN void level_full(float* v, uint8_t* cs, const Hot h)
{
    pass_full<A, S, D0, 0, D0, D1, D2, CUBIC, COMP>(v, cs, h);
    __syncthreads();
    pass_full<A, S, D1, 1, D0, D1, D2, CUBIC, COMP>(v, cs, h);
    __syncthreads();
    pass_full<A, S, D2, 2, D0, D1, D2, CUBIC, COMP>(v, cs, h);
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Multi-dimensional interpolation (Sec. 5.1.2): the level's points are taken
// in three phases by the number of their coordinates that are odd multiples
// of S (1, 2, then 3); a point is interpolated along each of its odd dims
// with that dim's 1D stencil, and the prediction is the mean of the
// interpolations of the highest order (cubic 3, quadratic 2, linear 1,
// copy 0), summed in increasing dim order: one as is, two times 0.5, three
// divided by 3.  Run-time extents; one block barrier per phase.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int stencil_order(bool cubic, bool have_l3, bool have_r, bool have_r3)
{
    if (!have_r) return have_l3 ? 1 : 0;
    if (!cubic) return 1;
    if (have_l3 && have_r3) return 3;
    return (have_l3 || have_r3) ? 2 : 1;
}

template <int A, bool COMP>
__device__ __noinline__ void level_md(int S, bool cubic, float* v, uint8_t* cs, const Hot h, int e0, int e1, int e2)
{
    using Lw = Lay<A>;
    constexpr int CX = COMP ? Lw::CXC : Lw::CXD, CY = COMP ? Lw::CYC : Lw::CYD;
    const int e[3] = {e0, e1, e2};
    const int act = (e0 > 0 ? 1 : 0) | (e1 > 0 ? 2 : 0) | (e2 > 0 ? 4 : 0);  // extent 0: inactive dim
    for (int k = 1; k <= 3; ++k) {
        for (int m = 1; m < 8; ++m) {
            if (__popc(m) != k || (m & ~act)) continue;
            int n[3];
#pragma unroll
            for (int d = 0; d < 3; ++d)
                n[d] = ((m >> d) & 1) ? (e[d] >= S ? (e[d] - S) / (2 * S) + 1 : 0) : e[d] / (2 * S) + 1;
            const int total = n[0] * n[1] * n[2];
            for (int i = threadIdx.x; i < total; i += blockDim.x) {
                const int j2 = i % n[2], r = i / n[2];
                const int j1 = r % n[1], j0 = r / n[1];
                const int jj[3] = {j0, j1, j2};
                int c[3];
#pragma unroll
                for (int d = 0; d < 3; ++d) c[d] = ((m >> d) & 1) ? (2 * jj[d] + 1) * S : 2 * jj[d] * S;
                const int vi = c[0] * Lw::PY + c[1] * Lw::PX + c[2];
                float p[3];
                int o[3];
                int best = -1;
#pragma unroll
                for (int d = 0; d < 3; ++d) {
                    p[d] = 0.0f;
                    o[d] = -1;
                    if (!((m >> d) & 1)) continue;
                    const int st = (d == 0 ? Lw::PY : (d == 1 ? Lw::PX : 1)) * S;
                    const bool have_r = c[d] + S <= e[d], have_l3 = c[d] >= 3 * S, have_r3 = c[d] + 3 * S <= e[d];
                    const float b = v[vi - st];
                    const float u = have_r ? v[vi + st] : 0.0f;
                    const float a = have_l3 ? v[vi - 3 * st] : 0.0f;
                    const float w = have_r3 ? v[vi + 3 * st] : 0.0f;
                    p[d] = predict(cubic, have_l3, have_r, have_r3, a, b, u, w);
                    o[d] = stencil_order(cubic, have_l3, have_r, have_r3);
                    best = o[d] > best ? o[d] : best;
                }
                float sum = 0.0f;
                int cnt = 0;
#pragma unroll
                for (int d = 0; d < 3; ++d)
                    if (o[d] == best) {
                        sum = cnt == 0 ? p[d] : __fadd_rn(sum, p[d]);
                        ++cnt;
                    }
                const float pr = cnt == 1 ? sum : (cnt == 2 ? __fmul_rn(sum, 0.5f) : __fdiv_rn(sum, 3.0f));
                const int ci = c[0] * CY + c[1] * CX + c[2];
                if constexpr (COMP)
                    v[vi] = point_compress(h, v[vi], pr, cs + ci);
                else
                    v[vi] = point_decompress<A>(h, cs[ci], pr, vi);
            }
        }
        __syncthreads();
    }
}

// The multi-dimensional scheme on a whole 3D tile: the points whose odd
// dims are the set M, everything known at compile time (counts, divisions,
// stencil cases: along an odd dim with NO odd positions, position j has
// f(c-3S) when j >= 1 and f(c+3S) when j <= NO - 2; f(c+S) always).
template <int A, int S, int M, bool CUBIC, bool COMP>
__device__ __forceinline__ void md_set_full(float* v, uint8_t* cs, const Hot h)
{
    using Lw = Lay<A>;
    constexpr int CX = COMP ? Lw::CXC : Lw::CXD, CY = COMP ? Lw::CYC : Lw::CYD;
    constexpr int NO = A / (2 * S), NE = A / (2 * S) + 1;
    constexpr int N0 = (M & 1) ? NO : NE, N1 = (M & 2) ? NO : NE, N2 = (M & 4) ? NO : NE;
    constexpr int TOTAL = N0 * N1 * N2;
    for (int i = threadIdx.x; i < TOTAL; i += blockDim.x) {
        const int j2 = i % N2, r = i / N2;
        const int j1 = r % N1, j0 = r / N1;
        const int c0 = (M & 1) ? (2 * j0 + 1) * S : 2 * j0 * S;
        const int c1 = (M & 2) ? (2 * j1 + 1) * S : 2 * j1 * S;
        const int c2 = (M & 4) ? (2 * j2 + 1) * S : 2 * j2 * S;
        const int vi = c0 * Lw::PY + c1 * Lw::PX + c2;
        const int jd[3] = {j0, j1, j2};
        float p[3];
        int o[3];
        int best = -1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p[d] = 0.0f;
            o[d] = -1;
            if (!((M >> d) & 1)) continue;
            const int st = (d == 0 ? Lw::PY : (d == 1 ? Lw::PX : 1)) * S;
            const bool l3 = CUBIC && jd[d] >= 1, r3 = CUBIC && jd[d] <= NO - 2;
            const float b = v[vi - st], u = v[vi + st];
            const float a = l3 ? v[vi - 3 * st] : 0.0f;
            const float w = r3 ? v[vi + 3 * st] : 0.0f;
            p[d] = predict(CUBIC, l3, true, r3, a, b, u, w);
            o[d] = !CUBIC ? 1 : ((l3 && r3) ? 3 : ((l3 || r3) ? 2 : 1));
            best = o[d] > best ? o[d] : best;
        }
        float sum = 0.0f;
        int cnt = 0;
#pragma unroll
        for (int d = 0; d < 3; ++d)
            if (o[d] == best) {
                sum = cnt == 0 ? p[d] : __fadd_rn(sum, p[d]);
                ++cnt;
            }
        const float pr = cnt == 1 ? sum : (cnt == 2 ? __fmul_rn(sum, 0.5f) : __fdiv_rn(sum, 3.0f));
        const int ci = c0 * CY + c1 * CX + c2;
        if constexpr (COMP)
            v[vi] = point_compress(h, v[vi], pr, cs + ci);
        else
            v[vi] = point_decompress<A>(h, cs[ci], pr, vi);
    }
}

template <int A, int S, bool CUBIC, bool COMP>
__device__ HI_LEVEL_FN void level_md_full(float* v, uint8_t* cs, const Hot h)
{
    md_set_full<A, S, 1, CUBIC, COMP>(v, cs, h);  // one odd dim
    md_set_full<A, S, 2, CUBIC, COMP>(v, cs, h);
    md_set_full<A, S, 4, CUBIC, COMP>(v, cs, h);
    __syncthreads();
    md_set_full<A, S, 3, CUBIC, COMP>(v, cs, h);  // two
    md_set_full<A, S, 5, CUBIC, COMP>(v, cs, h);
    md_set_full<A, S, 6, CUBIC, COMP>(v, cs, h);
    __syncthreads();
    md_set_full<A, S, 7, CUBIC, COMP>(v, cs, h);  // three
    __syncthreads();
}

// sel = 2 * perm + cubic; perm: 0 (0,1,2) 1 (0,2,1) 2 (1,0,2) 3 (1,2,0) 4 (2,0,1) 5 (2,1,0);
// 12 / 13: the multi-dimensional scheme with linear / cubic splines
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
    case 11: level_full<A, S, 2, 1, 0, true, COMP>(v, cs, h); break;
    case 12: level_md_full<A, S, false, COMP>(v, cs, h); break;
    default: level_md_full<A, S, true, COMP>(v, cs, h); break;
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
    if (lv.interp == HI_MD_LINEAR) return 12;
    if (lv.interp == HI_MD_CUBIC) return 13;
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

template <int A, int S, int D, bool COMP, int ED>
__device__ __forceinline__ void pass_spline(bool cubic, float* v, uint8_t* cs, const Hot h, int stq, int str, int nq,
                                            int nr, int ed)
{
    if (cubic)
        pass_any<A, S, D, true, COMP, ED, true>(v, cs, h, stq, str, nq, nr, ed);
    else
        pass_any<A, S, D, false, COMP, ED, true>(v, cs, h, stq, str, nq, nr, ed);
}

template <int A, int S, int D, bool COMP>
__device__ __forceinline__ void pass_dispatch(bool cubic, float* v, uint8_t* cs, const Hot h, int stq, int str,
                                              int nq, int nr, int ed)
{
    // one run-time instantiation for every extent: instantiations for the
    // common extents A and A - 1 ran the same instruction count and cost
    // more instruction fetch
    pass_spline<A, S, D, COMP, 0>(cubic, v, cs, h, stq, str, nq, nr, ed);
}

template <int A, int LV, bool COMP>
__device__ HI_LEVEL_FN void level_ragged(const hi_level lv, float* v, uint8_t* cs, const Hot h, int e0, int e1,
                                          int e2)
{
    constexpr int S = 1 << LV;
    if (lv.interp == HI_MD_LINEAR || lv.interp == HI_MD_CUBIC) {
        level_md<A, COMP>(S, lv.interp == HI_MD_CUBIC, v, cs, h, e0, e1, e2);
        return;
    }
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
// Tiles that TMA cannot stage (a row pitch that is not a multiple of 16
// bytes, an unaligned base).
//
// 16-byte aligned base: a row of e2 + 1 floats starting at float offset s
// is read as the aligned float4 chunks that cover it (one lane per chunk,
// LPR lanes per row, U rows per lane in flight) and realigned against the
// next lane's chunk; each lane stores one aligned float4 of the
// shared-memory row (floats past e2 land in the row's padding).  Chunks that
// would reach past the field's end are read float by float.
// Otherwise: a warp per row, 4-byte cp.async per float.
// The caller synchronises.
template <int A>
__device__ void load_tile_plain(float* v, const float* __restrict__ x, const FieldGeo& g, const TileInfo& ti)
{
    using Lw = Lay<A>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int e2 = ti.e[2];
    const int w1 = ti.e[1] + 1, rows = (ti.e[0] + 1) * w1;
    if ((reinterpret_cast<uintptr_t>(x) & 15u) == 0) {
        constexpr int LPR = (A >= 32) ? 16 : 8;
        constexpr int RPS = 32 / LPR;
        constexpr int U = 3;
        static_assert((3 + A) / 4 + 1 <= LPR, "row chunks");
        static_assert((A / 4) * 4 + 3 < Lw::PX, "the last chunk of a row stays in its padding");
        const int j = lane % LPR, sub = lane / LPR;
        const float inv_w1 = 1.0f / (float)w1;
        for (int r0 = warp * RPS + sub; r0 - sub < rows; r0 += nw * RPS * U) {
            float4 cv[U];
            int dv[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int r = r0 + u * nw * RPS;
                cv[u] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                dv[u] = 0;
                if (r < rows) {
                    const int c0 = (int)(((float)r + 0.5f) * inv_w1), c1 = r - c0 * w1;
                    const int64_t si = ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2];
                    const int d = (int)(si & 3);
                    dv[u] = d;
                    const int64_t ci = si - d + 4 * j;  // first float of this lane's chunk
                    if (4 * j <= d + e2) {
                        if (ci + 4 <= g.N) {
                            cv[u] = __ldg(reinterpret_cast<const float4*>(x + ci));
                        } else {
                            cv[u].x = x[ci];
                            if (ci + 1 < g.N) cv[u].y = x[ci + 1];
                            if (ci + 2 < g.N) cv[u].z = x[ci + 2];
                        }
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                float4 nx;
                nx.x = __shfl_down_sync(0xffffffffu, cv[u].x, 1);
                nx.y = __shfl_down_sync(0xffffffffu, cv[u].y, 1);
                nx.z = __shfl_down_sync(0xffffffffu, cv[u].z, 1);
                const int r = r0 + u * nw * RPS;
                if (r < rows && 4 * j <= e2) {
                    const int c0 = (int)(((float)r + 0.5f) * inv_w1), c1 = r - c0 * w1;
                    const float4 a = cv[u];
                    const int d = dv[u];
                    float4 o;
                    o.x = d == 0 ? a.x : (d == 1 ? a.y : (d == 2 ? a.z : a.w));
                    o.y = d == 0 ? a.y : (d == 1 ? a.z : (d == 2 ? a.w : nx.x));
                    o.z = d == 0 ? a.z : (d == 1 ? a.w : (d == 2 ? nx.x : nx.y));
                    o.w = d == 0 ? a.w : (d == 1 ? nx.x : (d == 2 ? nx.y : nx.z));
                    *reinterpret_cast<float4*>(v + c0 * Lw::PY + c1 * Lw::PX + 4 * j) = o;
                }
            }
        }
        return;
    }
    const int64_t rs = g.n[2], ps = g.n[1] * g.n[2];
    const float* base = x + ((int64_t)ti.o[0] * g.n[1] + ti.o[1]) * g.n[2] + ti.o[2];
    int c0 = warp / w1, c1 = warp - (warp / w1) * w1;
    for (int rr = warp; rr < rows; rr += nw) {
        const float* src = base + c0 * ps + c1 * rs;
        float* dst = v + c0 * Lw::PY + c1 * Lw::PX;
        for (int c2 = lane; c2 <= e2; c2 += 32) cp_async4(dst + c2, src + c2);
        c1 += nw;
        while (c1 >= w1) c1 -= w1, ++c0;
    }
    cp_async_wait_all();
}

// Codes of such a tile.  A row of e2 + 1 bytes starting at an arbitrary
// byte address is read as the aligned 4-byte words that cover it (one lane
// per word, LPR lanes per row, U rows per lane in flight) and realigned with
// a funnel shift against the next lane's word; each lane stores one aligned
// word of the shared-memory row (the bytes past e2 land in the row's
// padding).  Words that would reach outside [codes, codes + N) are read
// byte by byte.
template <int A>
__device__ void load_codes_plain(uint8_t* cs, const uint8_t* __restrict__ codes, const FieldGeo& g,
                                 const TileInfo& ti)
{
    using Lw = Lay<A>;
    constexpr int LPR = (A >= 32) ? 16 : 8;  // lanes per row: (3 + A) / 4 + 1 words at most
    constexpr int RPS = 32 / LPR;            // rows per warp step
    constexpr int U = 4;                     // warp steps in flight
    static_assert((3 + A) / 4 + 1 <= LPR, "row words");
    static_assert((A / 4) * 4 + 3 < Lw::CXD, "the last word of a row stays in its padding");
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int j = lane % LPR, sub = lane / LPR;
    const int e2 = ti.e[2];
    const int w1 = ti.e[1] + 1, rows = (ti.e[0] + 1) * w1;
    const float inv_w1 = 1.0f / (float)w1;
    const uintptr_t lo = reinterpret_cast<uintptr_t>(codes), hi = lo + (uintptr_t)g.N;
    for (int r0 = warp * RPS + sub; r0 - sub < rows; r0 += nw * RPS * U) {
        uint32_t wv[U];
        uint32_t dv[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int r = r0 + u * nw * RPS;
            wv[u] = 0u;
            dv[u] = 0u;
            if (r < rows) {
                const int c0 = (int)(((float)r + 0.5f) * inv_w1), c1 = r - c0 * w1;
                const uintptr_t a = lo + (uintptr_t)(((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] +
                                                     ti.o[2]);
                const uint32_t d = (uint32_t)(a & 3u);
                dv[u] = d;
                const uintptr_t w = a - d + 4u * (uint32_t)j;
                if (4 * j <= (int)d + e2) {
                    if (w >= lo && w + 4 <= hi) {
                        wv[u] = __ldg(reinterpret_cast<const uint32_t*>(w));
                    } else {
                        uint32_t t = 0;
                        for (int b = 0; b < 4; ++b)
                            if (w + b >= lo && w + b < hi) t |= (uint32_t)(*reinterpret_cast<const uint8_t*>(w + b)) << (8 * b);
                        wv[u] = t;
                    }
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint32_t nxt = __shfl_down_sync(0xffffffffu, wv[u], 1);
            const int r = r0 + u * nw * RPS;
            if (r < rows && 4 * j <= e2) {
                const int c0 = (int)(((float)r + 0.5f) * inv_w1), c1 = r - c0 * w1;
                const uint32_t word = __funnelshift_r(wv[u], j + 1 < LPR ? nxt : 0u, 8 * dv[u]);
                *reinterpret_cast<uint32_t*>(cs + c0 * Lw::CYD + c1 * Lw::CXD + 4 * j) = word;
            }
        }
    }
}

// L2 prefetch of the rows of a tile that the plain loaders will read: the
// first and last element of each row (elem bytes each).
template <int A>
__device__ __forceinline__ void prefetch_rows_l2(const void* base, int elem, const FieldGeo& g, const TileInfo& ti)
{
    const int w1 = ti.e[1] + 1, rows = (ti.e[0] + 1) * w1;
    const char* b = static_cast<const char*>(base);
    for (int r = threadIdx.x; r < rows; r += blockDim.x) {
        const int c0 = r / w1, c1 = r - c0 * w1;
        const int64_t i = ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2];
        prefetch_l2(b + i * elem);
        prefetch_l2(b + (i + ti.e[2]) * elem);
    }
}

// Queue position with the field's shell (its last blocks along each dim,
// the ragged tiles of most fields) taken first, then the interior: the slow
// tiles start early instead of forming the launch's tail.
__device__ __forceinline__ int shell_first(const FieldGeo& g, int pos)
{
    const int n_shell = g.ntiles - g.ni[0] * g.ni[1] * g.ni[2];
    return pos < n_shell ? pos + (g.ntiles - n_shell) : pos - n_shell;
}

// L2 prefetch of the box of the tile at queue position `tile`.
__device__ __forceinline__ void tma_l2_prefetch(const CUtensorMap* map, const FieldGeo& g, int tile, int A)
{
    int t[3];
    tile_coords(g, tile, t);
    tma_prefetch_3d(map, t[2] * A, t[1] * A, t[0] * A);
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

// Outliers of NW 4-byte code words per lane (all lanes of the warp call
// it): zm[j] has 0x80 in each byte of word j whose code is 0; the codes
// stand at float offsets vi0 + 4 j + byte in the tile.  The warp reserves its
// slots with one atomic (a prefix sum over the lanes' counts) and each lane
// writes its own outliers.
template <int A, int NW>
__device__ __forceinline__ void outliers_append_words(const uint32_t* zm, int vi0, const float* v, hi_header* hdr,
                                                      uint32_t* out_idx, float* out_val, uint64_t out_cap,
                                                      const FieldGeo& g, const int o[3])
{
    const int lane = threadIdx.x & 31;
    int cnt = 0;
#pragma unroll
    for (int j = 0; j < NW; ++j) cnt += __popc(zm[j]);
    int incl = cnt;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += t;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31) base = atomicAdd(reinterpret_cast<unsigned long long*>(&hdr->n_outliers), (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned long long pos = base + (unsigned long long)(incl - cnt);
    bool over = false;
#pragma unroll
    for (int j = 0; j < NW; ++j) {
        uint32_t m = zm[j];
        while (m) {
            const int bit = __ffs(m) - 1;  // 7, 15, 23 or 31
            m &= m - 1;
            const int vi = vi0 + 4 * j + (bit >> 3);
            if (pos < out_cap) {
                out_idx[pos] = (uint32_t)global_index<A>(g, o, vi);
                out_val[pos] = v[vi];
            } else {
                over = true;
            }
            ++pos;
        }
    }
    if (over) set_status(&hdr->status, HI_ECAPACITY);
}

// Histogram: codes 120..135 (the bulk at any practical error bound) go to
// per-thread 16-bit counters laid out bin-major, so that a warp's updates hit
// 32 consecutive half-words (no bank conflict, no atomics); other codes go
// to shared-memory atomics.  Folded into the CTA histogram at kernel end.
constexpr int kHistLo = 120, kHistBins = 16;

// Histogram of tiles of A <= 16: codes 126..129 (the bulk at practical error
// bounds) in the four bytes of one register per thread, folded into the CTA
// histogram at the end of every tile (a thread counts fewer than 256 codes of
// a tile); other codes by a predicated shared-memory reduction, no branch.
constexpr uint32_t kHotLo = 126;

// One code: the hot bins add 1 << 8 (code - 126) to hacc (0 for codes past
// 129: the funnel shift clamps at 32); codes below 126 wrap to a shift past
// 32 as well; every code outside the hot bins is added to s_hist by a
// predicated shared-memory reduction (no branch).  `valid` false counts
// nothing.
__device__ __forceinline__ void hist_hot(uint32_t code, bool valid, uint32_t& hacc, uint32_t* s_hist)
{
    const uint32_t sh = code * 8u - 8u * kHotLo;
    hacc += valid ? __funnelshift_lc(0u, 1u, sh) : 0u;  // 1 << sh; 0 for sh >= 32
    asm volatile(
        "{\n\t.reg .pred pv, pc;\n\t"
        "setp.ne.u32 pv, %2, 0;\n\t"
        "setp.ge.and.u32 pc, %0, 32, pv;\n\t"
        "@pc red.shared.add.u32 [%1], 1;\n\t}" ::"r"(sh),
        "r"(smem_addr(s_hist) + 4u * code), "r"((uint32_t)valid)
        : "memory");
}

// The four codes of a word (all valid): one shift amount, one hot add and
// one predicated reduction per code.
__device__ __forceinline__ void hist_hot4(uint32_t w, uint32_t& hacc, uint32_t s_base)
{
    uint32_t sh[4], ad[4];
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t c = __byte_perm(w, 0u, 0x4440u | (uint32_t)b);
        ad[b] = s_base + 4u * c;
        sh[b] = 8u * c - 8u * kHotLo;
        hacc += __funnelshift_lc(0u, 1u, sh[b]);
    }
    asm volatile(
        "{\n\t.reg .pred p0, p1, p2, p3;\n\t"
        "setp.ge.u32 p0, %0, 32;\n\t"
        "setp.ge.u32 p1, %1, 32;\n\t"
        "setp.ge.u32 p2, %2, 32;\n\t"
        "setp.ge.u32 p3, %3, 32;\n\t"
        "@p0 red.shared.add.u32 [%4], 1;\n\t"
        "@p1 red.shared.add.u32 [%5], 1;\n\t"
        "@p2 red.shared.add.u32 [%6], 1;\n\t"
        "@p3 red.shared.add.u32 [%7], 1;\n\t}" ::"r"(sh[0]),
        "r"(sh[1]), "r"(sh[2]), "r"(sh[3]), "r"(ad[0]), "r"(ad[1]), "r"(ad[2]), "r"(ad[3])
        : "memory");
}

// The four codes of a word, counted only when `valid`.
__device__ __forceinline__ void hist_hot4(uint32_t w, bool valid, uint32_t& hacc, uint32_t* s_hist)
{
    if (valid) hist_hot4(w, hacc, smem_addr(s_hist));
}

// Fold the register counters into the CTA histogram and clear them (whole warps).
__device__ __forceinline__ void hist_hot_flush(uint32_t& hacc, uint32_t* s_hist)
{
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t n = __reduce_add_sync(0xffffffffu, (hacc >> (8 * b)) & 0xffu);
        if ((threadIdx.x & 31) == 0 && n) atomicAdd(&s_hist[kHotLo + b], n);
    }
    hacc = 0;
}

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
// Batches: work items over the concatenated tile lists of many fields
// ---------------------------------------------------------------------------
// The field whose work items [start[f], start[f+1]) contain w (fields
// without work items are skipped).
__device__ __forceinline__ int find_field(const uint32_t* __restrict__ start, int n, uint32_t w)
{
    int lo = 0, hi = n;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(start + mid) <= w)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// Work item w -> (field, position in the field's queue order).  The head
// tiles of every field (its whole 3D tiles) come first, then the rest of
// every field: the CTAs in flight mostly run one kind of pass code.
__device__ __forceinline__ int batch_locate(const BatchField* __restrict__ fields,
                                            const uint32_t* __restrict__ head_start,
                                            const uint32_t* __restrict__ shell_start, int n, uint32_t total_head,
                                            uint32_t w, int* pos)
{
    if (w < total_head) {
        const int f = find_field(head_start, n, w);
        *pos = (int)(w - __ldg(head_start + f));
        return f;
    }
    const uint32_t w2 = w - total_head;
    const int f = find_field(shell_start, n, w2);
    *pos = (int)(fields[f].nint + (w2 - __ldg(shell_start + f)));
    return f;
}

// Shared-memory footprint of the two kernels and the persistent launch.
template <int A>
size_t compress_smem_t(int b0, bool dbuf, int threads)
{
    // 16-bit per-thread histogram counters only where the register counters
    // of hist_hot could overflow within a tile (A = 32)
    return (dbuf ? 2 : 1) * (size_t)vbuf_bytes<A>(b0) + (size_t)round128(b0 * Lay<A>::P * Lay<A>::CXC) +
           (A > 16 ? (size_t)kHistBins * threads * sizeof(uint16_t) : 0);
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

// Resident CTAs per SM of a kernel at a launch shape, asked of the runtime
// once per (device, kernel, threads, shared memory) and kept: the queries
// cost more host time than a launch.
struct OccKey {
    int dev;
    const void* kern;
    int threads;
    size_t smem;
    bool operator<(const OccKey& o) const
    {
        if (dev != o.dev) return dev < o.dev;
        if (kern != o.kern) return kern < o.kern;
        if (threads != o.threads) return threads < o.threads;
        return smem < o.smem;
    }
};

template <typename K>
static cudaError_t ctas_per_sm(K kern, int threads, size_t smem, int* per_sm)
{
    static std::mutex mu;
    static std::map<OccKey, int> cache;
    int dev = 0;
    cudaError_t err = cudaGetDevice(&dev);
    if (err != cudaSuccess) return err;
    const OccKey key{dev, reinterpret_cast<const void*>(kern), threads, smem};
    std::lock_guard<std::mutex> lock(mu);
    auto it = cache.find(key);
    if (it != cache.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    err = set_max_smem(kern, smem);
    if (err != cudaSuccess) return err;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, kern, threads, smem);
    if (err != cudaSuccess) return err;
    cache[key] = *per_sm;
    return cudaSuccess;
}

template <typename K>
static cudaError_t persistent_grid(K kern, int threads, size_t smem, int num_sms, int ntiles, int max_ctas, int* grid)
{
    int per_sm = 0;
    cudaError_t err = ctas_per_sm(kern, threads, smem, &per_sm);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    int g = per_sm * num_sms;
    if (g > ntiles) g = ntiles;
    if (max_ctas > 0 && g > max_ctas) g = max_ctas;
    *grid = g > 0 ? g : 1;
    return cudaSuccess;
}

}  // namespace hi
