// hi_compress_tile.cuh -- one tile of the fused predict + quantize step
// (Sec. 5.1.1-5.1.2, Sec. 5.2.1), shared by the single-field kernel and the
// batched kernel: the level passes over a staged tile, then the epilogue that
// stores the owned codes and anchors, appends the outliers and counts the
// histogram.
#pragma once

#include "hi_passes.cuh"

namespace hi {

// Reordered-sequence store of one tile row (Sec. 5.2.2, Eq. 3): the A codes
// of row (x, y), columns z0 .. z0 + A - 1 (z0 a multiple of A), 4 to a word
// in w.  On the stride-2^l subgrid the row (x >> l, y >> l) holds A >> l of
// them from column z0 >> l: if x >> l or y >> l is odd all are on level l,
// at consecutive places; otherwise the odd columns are on level l, at
// consecutive places, and the even ones go on to level l + 1; on level
// log2 A the one left is an anchor.  A place is prefix[l] (the coarser
// points) + the row-major rank on the subgrid - the all-even points before
// it.  Callers take this path only where every run starts at a multiple of
// its length, so each run is one aligned store.  (seq_store_tile below runs
// it for the rows of tiles that are not whole.)
template <int N>
__device__ __forceinline__ void seq_store_run(uint8_t* p, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3)
{
    if constexpr (N == 16)
        *reinterpret_cast<uint4*>(p) = make_uint4(v0, v1, v2, v3);
    else if constexpr (N == 8)
        *reinterpret_cast<uint2*>(p) = make_uint2(v0, v1);
    else if constexpr (N == 4)
        *reinterpret_cast<uint32_t*>(p) = v0;
    else if constexpr (N == 2)
        *reinterpret_cast<uint16_t*>(p) = (uint16_t)v0;
    else
        *p = (uint8_t)v0;
}

template <int A, int l>
__device__ __forceinline__ void seq_store_level(uint8_t* __restrict__ seq, const SeqGeo& sg, uint32_t x, uint32_t y,
                                                uint32_t z0, uint32_t v0, uint32_t v1, uint32_t v2, uint32_t v3)
{
    constexpr int L = (A == 16) ? 4 : 3;
    constexpr int N = A >> l;  // codes of the row on this subgrid
    const uint32_t xs = x >> l, ys = y >> l, zs = z0 >> l;
    const uint32_t rank = (xs * sg.D1[l] + ys) * sg.D2[l];
    if constexpr (l == L) {
        seq[rank + zs] = (uint8_t)v0;  // the anchors come first: prefix 0
    } else {
        uint32_t base = sg.prefix[l] + rank - ((xs + 1u) >> 1) * sg.H12[l];
        if ((xs & 1u) == 0) base -= ((ys + 1u) >> 1) * sg.H2[l];
        if ((xs | ys) & 1u) {
            seq_store_run<N>(seq + base + zs, v0, v1, v2, v3);
            return;
        }
        uint32_t o0, o1 = 0u, e0, e1 = 0u;  // odd and even columns, in order
        if constexpr (N == 16) {
            o0 = __byte_perm(v0, v1, 0x7531), o1 = __byte_perm(v2, v3, 0x7531);
            e0 = __byte_perm(v0, v1, 0x6420), e1 = __byte_perm(v2, v3, 0x6420);
        } else if constexpr (N == 8) {
            o0 = __byte_perm(v0, v1, 0x7531), e0 = __byte_perm(v0, v1, 0x6420);
        } else if constexpr (N == 4) {
            o0 = __byte_perm(v0, 0u, 0x31), e0 = __byte_perm(v0, 0u, 0x20);
        } else {
            o0 = v0 >> 8, e0 = v0;
        }
        seq_store_run<N / 2>(seq + base + (zs >> 1), o0, o1, 0u, 0u);
        seq_store_level<A, l + 1>(seq, sg, x, y, z0, e0, e1, 0u, 0u);
    }
}

template <int A>
__device__ __forceinline__ void seq_store_row(uint8_t* __restrict__ seq, const SeqGeo& sg, uint32_t x, uint32_t y,
                                              uint32_t z0, const uint32_t* w)
{
    static_assert(A == 8 || A == 16, "rows of 8 or 16 codes");
    seq_store_level<A, 0>(seq, sg, x, y, z0, w[0], w[1], A == 16 ? w[2] : 0u, A == 16 ? w[3] : 0u);
}

// The codes of columns k 2^l of a row (ODD: odd k only), packed 4 to a word.
template <int A, int l, bool ODD>
__device__ __forceinline__ void seq_gather(const uint32_t* w, uint32_t* o)
{
    constexpr int M = A >> l, K = ODD ? M / 2 : M;
#pragma unroll
    for (int j = 0; j < 4; ++j) o[j] = 0u;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const int byte = (ODD ? 2 * j + 1 : j) << l;
        o[j >> 2] |= ((w[byte >> 2] >> (8 * (byte & 3))) & 0xffu) << (8 * (j & 3));
    }
}

// Level l of a whole tile's sequence store: the rows whose coordinates are
// multiples of 2^l, the M = A >> l codes of each at columns k 2^l.  Rows
// with an odd coordinate on this subgrid are one run each and come first,
// then the all-even rows, whose odd columns are one run (their even ones
// are level l + 1's rows): each warp issues one kind of store, save at the
// boundary.
template <int A, int l>
__device__ __forceinline__ void seq_level_pass(uint8_t* __restrict__ seq, const SeqGeo& sg, const TileInfo& ti,
                                               const uint8_t* cs)
{
    using Lw = Lay<A>;
    constexpr int M = A >> l, H = M / 2;
    constexpr int n_first = H * M, n_odd = M * M - H * H;
    const uint32_t zs = (uint32_t)ti.o[2] >> l;
    for (int r = threadIdx.x; r < M * M; r += blockDim.x) {
        int a, b;
        if (r < n_first) {  // odd a, any b
            a = 2 * (r / M) + 1, b = r - (r / M) * M;
        } else {
            const int j = r - (r < n_odd ? n_first : n_odd);
            a = 2 * (j / H), b = 2 * (j - (j / H) * H) + (r < n_odd ? 1 : 0);
        }
        const int c0 = a << l, c1 = b << l;
        const uint32_t* src = reinterpret_cast<const uint32_t*>(cs + c0 * Lw::CYC + c1 * Lw::CXC);
        uint32_t w[A / 4];
#pragma unroll
        for (int j = 0; j < A / 4; ++j) w[j] = src[j];
        const uint32_t xs = ((uint32_t)ti.o[0] + c0) >> l, ys = ((uint32_t)ti.o[1] + c1) >> l;
        uint32_t base = sg.prefix[l] + (xs * sg.D1[l] + ys) * sg.D2[l] - ((xs + 1u) >> 1) * sg.H12[l];
        if ((xs & 1u) == 0) base -= ((ys + 1u) >> 1) * sg.H2[l];
        uint32_t o[4];
        if (r < n_odd) {
            seq_gather<A, l, false>(w, o);
            seq_store_run<M>(seq + base + zs, o[0], o[1], o[2], o[3]);
        } else {
            seq_gather<A, l, true>(w, o);
            seq_store_run<H>(seq + base + (zs >> 1), o[0], o[1], o[2], o[3]);
        }
    }
}

// A tile's owned codes (staged in cs) to their places in the sequence.
// Whole tiles (own0 = own1 = A) level by level; the others row by row.
template <int A>
__device__ __forceinline__ void seq_store_tile(uint8_t* __restrict__ seq, const SeqGeo& sg, const TileInfo& ti,
                                               const uint8_t* cs, int own0, int own1)
{
    using Lw = Lay<A>;
    constexpr int L = (A == 16) ? 4 : 3;
    if (own0 == A && own1 == A) {
        seq_level_pass<A, 0>(seq, sg, ti, cs);
        seq_level_pass<A, 1>(seq, sg, ti, cs);
        seq_level_pass<A, 2>(seq, sg, ti, cs);
        if constexpr (L == 4) seq_level_pass<A, 3>(seq, sg, ti, cs);
        if (threadIdx.x == 0) {  // the anchor row's one code on level log2 A
            const uint32_t xs = (uint32_t)ti.o[0] >> L, ys = (uint32_t)ti.o[1] >> L, zs = (uint32_t)ti.o[2] >> L;
            seq[(xs * sg.D1[L] + ys) * sg.D2[L] + zs] = cs[0];
        }
    } else {
        for (int r = threadIdx.x; r < own0 * own1; r += blockDim.x) {
            const int c0 = r / own1, c1 = r - (r / own1) * own1;
            const uint32_t* src = reinterpret_cast<const uint32_t*>(cs + c0 * Lw::CYC + c1 * Lw::CXC);
            uint32_t w[A / 4];
#pragma unroll
            for (int j = 0; j < A / 4; ++j) w[j] = src[j];
            seq_store_row<A>(seq, sg, (uint32_t)(ti.o[0] + c0), (uint32_t)(ti.o[1] + c1), (uint32_t)ti.o[2], w);
        }
    }
}

// The tile's floats are in v (reconstructed in place), its codes are staged
// in cs; g, ti: the field and the tile; s_sel / s_lv: the level
// configuration; full_ok: the field may take the compile-time full-tile
// passes; out: a CompressOut or a reference to one in shared memory.  With
// SEQ the owned codes also go to the reordered sequence seq (constants sg),
// from cs after the epilogue; the caller takes SEQ only where every tile row
// is whole (n2 a multiple of A) and every run starts at a multiple of its
// length.
template <int A, bool SEQ = false, class Out>
__device__ __forceinline__ void compress_tile(const FieldGeo& g, const TileInfo& ti, float* v, uint8_t* cs,
                                              uint16_t* hc, uint32_t* s_hist, const int* s_sel,
                                              const hi_level* s_lv, const Hot h, bool full_ok, const Out& out,
                                              uint8_t* seq = nullptr, const SeqGeo* sg = nullptr)
{
    using Lw = Lay<A>;
    const int tid = threadIdx.x;
    const bool full = full_ok && ti.e[0] == A && ti.e[1] == A && ti.e[2] == A;
    if constexpr (HasFull<A>::value) {
        if (full)
            levels_full<A, TileGeom<A>::L - 1, true>(s_sel, v, cs, h);
        else
            levels_ragged<A, TileGeom<A>::L - 1, true>(s_lv, v, cs, h, ti);
    } else {
        levels_ragged<A, TileGeom<A>::L - 1, true>(s_lv, v, cs, h, ti);
    }
    const bool vec_ok = out.vec_ok, hist_on = out.hist_on;
    uint8_t* __restrict__ const codes = out.codes;
    float* __restrict__ const anchors = out.anchors;
    uint32_t* __restrict__ const out_idx = out.out_idx;
    float* __restrict__ const out_val = out.out_val;
    const uint64_t out_cap = out.out_cap;
    float* __restrict__ const recon_g = out.recon;
    hi_header* __restrict__ const hdr = out.hdr;

    // ---- epilogue: owned codes, histogram and outliers; recon; anchors
    const int own0 = ti.own[0] + 1, own1 = ti.own[1] + 1, own2 = ti.own[2] + 1;
    const int rows = own0 * own1;
    constexpr bool kHot = A <= 16;  // register histogram (see hist_hot)
    uint32_t hacc = 0;
    const bool vec_codes = vec_ok && own2 == A && A >= 8;
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
                uint32_t zm[CH];  // 0x80 in each byte that is zero (exact, no borrow between bytes)
#pragma unroll
                for (int j = 0; j < CH; ++j)
                    zm[j] = act ? ~(((w[j] & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w[j]) & 0x80808080u : 0u;
                outliers_append_words<A, CH>(zm, c0 * Lw::PY + c1 * Lw::PX + ch * CH * 4, v, hdr, out_idx, out_val,
                                             out_cap, g, ti.o);
            }
            if (hist_on) {
                if constexpr (kHot) {
                    if (act) {
                        const uint32_t sb = smem_addr(s_hist);
#pragma unroll
                        for (int j = 0; j < CH; ++j) hist_hot4(w[j], hacc, sb);
                    }
                } else {
                    for (int b = 0; b < 4 * CH; ++b)
                        hist_count(hc, s_hist, (w[b >> 2] >> (8 * (b & 3))) & 0xff, act);
                }
            }
        }
    } else if ((own2 & 3) == 0 && own2 <= 32) {
        // rows of whole 4-code words that cannot go out as 16-byte vectors
        // (row pitch or base not 16-byte aligned): a word per thread step,
        // stored as one word where the address allows, else as 4 bytes
        const int wpr = own2 >> 2;
        const int items = rows * wpr;
        const float inv_wpr = 1.0f / (float)wpr, inv_own1 = 1.0f / (float)own1;
        for (int i0 = 0; i0 < items; i0 += blockDim.x) {
            const int i = i0 + tid;
            const bool act = i < items;
            const int ii = act ? i : 0;
            const int row = (int)(((float)ii + 0.5f) * inv_wpr), k = ii - row * wpr;
            const int c0 = (int)(((float)row + 0.5f) * inv_own1), c1 = row - c0 * own1;
            const int vi = c0 * Lw::PY + c1 * Lw::PX + 4 * k;
            const uint32_t w = *reinterpret_cast<const uint32_t*>(cs + c0 * Lw::CYC + c1 * Lw::CXC + 4 * k);
            const int64_t gi = ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + 4 * k;
            if (act) {
                uint8_t* dst = codes + gi;
                if ((reinterpret_cast<uintptr_t>(dst) & 3u) == 0) {
                    *reinterpret_cast<uint32_t*>(dst) = w;
                } else {
                    dst[0] = (uint8_t)w;
                    dst[1] = (uint8_t)(w >> 8);
                    dst[2] = (uint8_t)(w >> 16);
                    dst[3] = (uint8_t)(w >> 24);
                }
                if (recon_g) {
#pragma unroll
                    for (int b = 0; b < 4; ++b) recon_g[gi + b] = v[vi + b];
                }
            }
            const uint32_t z = (w - 0x01010101u) & ~w & 0x80808080u;
            if (__any_sync(0xffffffffu, act && z != 0)) {
                uint32_t zm[1];
                zm[0] = act ? ~(((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w) & 0x80808080u : 0u;
                outliers_append_words<A, 1>(zm, vi, v, hdr, out_idx, out_val, out_cap, g, ti.o);
            }
            if (hist_on) {
                if constexpr (kHot) {
                    hist_hot4(w, act, hacc, s_hist);
                } else {
                    for (int b = 0; b < 4; ++b) hist_count(hc, s_hist, (w >> (8 * b)) & 0xff, act);
                }
            }
        }
    } else if (own2 <= 32) {
        // rows that are not stored as vectors: lanes over the columns, two
        // rows per warp step when they are at most 16 wide
        const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
        const bool two = own2 <= 16;
        const int rpw = two ? 2 : 1;
        const int sub = two ? (lane >> 4) : 0, col = two ? (lane & 15) : lane;
        for (int r0 = warp * rpw; r0 < rows; r0 += nw * rpw) {
            const int row = r0 + sub;
            const bool act = row < rows && col < own2;
            const int rr = act ? row : 0, c2 = act ? col : 0;
            const int c0 = rr / own1, c1 = rr - c0 * own1;
            const int code = cs[c0 * Lw::CYC + c1 * Lw::CXC + c2];
            const int64_t gi = ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2;
            if (act) {
                codes[gi] = (uint8_t)code;
                if (recon_g) recon_g[gi] = v[c0 * Lw::PY + c1 * Lw::PX + c2];
            }
            if (hist_on) {
                if constexpr (kHot)
                    hist_hot((uint32_t)code, act, hacc, s_hist);
                else
                    hist_count(hc, s_hist, code, act);
            }
            outlier_append<A>(act && code == 0, c0 * Lw::PY + c1 * Lw::PX + c2, v, hdr, out_idx, out_val, out_cap,
                              g, ti.o);
        }
    } else {
        const int items = rows * own2;
        for (int i0 = 0; i0 < items; i0 += blockDim.x) {
            const int i = i0 + tid;
            const bool act = i < items;
            const int row = act ? i / own2 : 0, c2 = act ? i - row * own2 : 0;
            const int c0 = row / own1, c1 = row - c0 * own1;
            const int code = cs[c0 * Lw::CYC + c1 * Lw::CXC + c2];
            if (act) {
                const int64_t gi = ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2;
                codes[gi] = (uint8_t)code;
                if (recon_g) recon_g[gi] = v[c0 * Lw::PY + c1 * Lw::PX + c2];
            }
            if (hist_on) {
                if constexpr (kHot)
                    hist_hot((uint32_t)code, act, hacc, s_hist);
                else
                    hist_count(hc, s_hist, code, act);
            }
            outlier_append<A>(act && code == 0, c0 * Lw::PY + c1 * Lw::PX + c2, v, hdr, out_idx, out_val, out_cap,
                              g, ti.o);
        }
    }
    if constexpr (kHot) {
        if (hist_on) hist_hot_flush(hacc, s_hist);
    }
    if constexpr (SEQ) seq_store_tile<A>(seq, *sg, ti, cs, own0, own1);
    if (recon_g && vec_codes) {
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
}

// Every kHistFoldTiles tiles a CTA folds its 16-bit histogram counters into
// the shared histogram, before any of them can overflow: a thread counts at
// most ceil(33^3 / 64) + 16 codes of a tile.
constexpr int kHistFoldTiles = 64;

// Fold the calling thread's counters into s_hist and clear them (whole warps).
__device__ __forceinline__ void hist_fold(uint16_t* hc, uint32_t* s_hist)
{
    if (hc == nullptr) return;  // tiles of A <= 16 count in registers (hist_hot)
    const int tid = threadIdx.x;
    for (int k = 0; k < kHistBins; ++k) {
        const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)hc[k * blockDim.x + tid]);
        hc[k * blockDim.x + tid] = 0;
        if ((tid & 31) == 0 && c) atomicAdd(&s_hist[kHistLo + k], c);
    }
}

// Add the CTA's counts to hist_g and clear them, with no barrier of its own:
// the hot bins of each warp go out straight from a warp reduction; the
// shared bins are read after a barrier that followed their last update and
// are next updated after a later one.  (The shared bin of code 128 may hold
// a wrapped negative count, the anchors taken off; the sum in hist_g is
// exact modulo 2^32.)
__device__ __forceinline__ void hist_flush_to(uint16_t* hc, uint32_t* s_hist, uint32_t* hist_g)
{
    const int tid = threadIdx.x;
    for (int k = 0; hc != nullptr && k < kHistBins; ++k) {
        const uint32_t c = __reduce_add_sync(0xffffffffu, (uint32_t)hc[k * blockDim.x + tid]);
        hc[k * blockDim.x + tid] = 0;
        if ((tid & 31) == 0 && c) atomicAdd(&hist_g[kHistLo + k], c);
    }
    for (int i = tid; i < 256; i += blockDim.x) {
        const uint32_t c = s_hist[i];
        if (c) {
            atomicAdd(&hist_g[i], c);
            s_hist[i] = 0;
        }
    }
}

// Fold, add the CTA's histogram to hist_g and clear it (all threads).
__device__ __forceinline__ void hist_flush(uint16_t* hc, uint32_t* s_hist, uint32_t* hist_g)
{
    hist_fold(hc, s_hist);
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x) {
        const uint32_t c = s_hist[i];
        if (c) atomicAdd(&hist_g[i], c);
        s_hist[i] = 0;
    }
    __syncthreads();
}

}  // namespace hi
