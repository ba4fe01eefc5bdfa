// hi_interp.cu -- fused interpolation-predict + quantize kernel and its
// inverse, the level-by-level reconstruction (cuSZ-Hi, arXiv 2507.11165,
// Sec. 3.2, Sec. 5.1.1-5.1.2, Sec. 5.2.1).
//
// One CTA works through blocks ("tiles") of (A+1)^d points in a grid-strided
// loop.  A tile is staged in shared memory by one 3D TMA box load (or by
// plain loads when the field's strides do not meet the TMA rules), then every
// level (stride s = A/2 .. 1) runs its three 1D passes in the configured
// dimension sequence.  Within a pass each thread owns one whole line along
// the pass dimension: the line's already-known nodes (even multiples of s)
// slide through four registers, so every predicted point costs one new node
// load, one load of its own value and one store.  Predictions read values
// already reconstructed in shared memory (closed loop), so the decompressor
// repeats exactly the same arithmetic.
//
// Shared faces between tiles are computed by both tiles with identical
// results; only the owning tile (the one with the lower block index, or the
// last block for the field's upper face) writes codes, histogram counts,
// outliers and reconstructed values.
#include <cstdint>

#include "hi_device.cuh"
#include "hi_internal.h"

namespace hi {

constexpr int kOutCap = 1024;  // staged outliers per tile before the direct path

struct PassGeom {
    int d, q, r;      // pass dim and the two others
    int stq, str;     // strides of the other two dims (s or 2s)
    int nd;           // predicted points per line
    int nq, nr;       // lines along q and r
};

// a[i] for a runtime i in {0,1,2}, without indexing (keeps a[] in registers)
__device__ __forceinline__ int pick3(const int a[3], int i) { return i == 0 ? a[0] : (i == 1 ? a[1] : a[2]); }

__device__ __forceinline__ PassGeom pass_geom(const hi_level& lv, int p, int s, const int e[3])
{
    PassGeom pg;
    pg.d = lv.order[p];
    pg.q = (pg.d == 0) ? 1 : 0;
    pg.r = (pg.d == 2) ? 1 : 2;
    // dims refined earlier in this level step by s; later ones by 2s
    const int posq = (lv.order[0] == pg.q) ? 0 : ((lv.order[1] == pg.q) ? 1 : 2);
    const int posr = (lv.order[0] == pg.r) ? 0 : ((lv.order[1] == pg.r) ? 1 : 2);
    pg.stq = (posq < p) ? s : 2 * s;
    pg.str = (posr < p) ? s : 2 * s;
    const int ed = pick3(e, pg.d);
    pg.nd = (ed >= s) ? ((ed - s) / (2 * s) + 1) : 0;
    pg.nq = pick3(e, pg.q) / pg.stq + 1;
    pg.nr = pick3(e, pg.r) / pg.str + 1;
    return pg;
}

template <int A>
__device__ __forceinline__ int vpitch(int d)
{
    using TG = TileGeom<A>;
    return d == 0 ? TG::PY : (d == 1 ? TG::PX : 1);
}

template <int A>
__device__ __forceinline__ int cpitch(int d)
{
    using TG = TileGeom<A>;
    return d == 0 ? TG::CY : (d == 1 ? TG::CX : 1);
}

// Warp-aggregated histogram update: lanes with equal codes add once.
__device__ __forceinline__ void hist_add(uint32_t* s_hist, int code, bool valid, int lane)
{
    const int key = valid ? code : 256;
    const unsigned m = __match_any_sync(0xffffffffu, key);
    if (valid && lane == __ffs(m) - 1) atomicAdd(&s_hist[code], (uint32_t)__popc(m));
}

// Global linear index of a local shared-memory float offset.
template <int A>
__device__ __forceinline__ int64_t global_index(const FieldGeo& g, const int o[3], int vi)
{
    using TG = TileGeom<A>;
    const int c0 = vi / TG::PY;
    const int rem = vi - c0 * TG::PY;
    const int c1 = rem / TG::PX;
    const int c2 = rem - c1 * TG::PX;
    return ((int64_t)(o[0] + c0) * g.n[1] + (o[1] + c1)) * g.n[2] + (o[2] + c2);
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
    for (int d = 0; d < 3; ++d) {
        ti.o[d] = t[d] * A;
        const int rem = (int)(g.n[d] - 1 - ti.o[d]);
        ti.e[d] = (g.n[d] == 1) ? 0 : (rem < A ? rem : A);
        ti.own[d] = (t[d] == g.nb[d] - 1) ? ti.e[d] : A - 1;
    }
    return ti;
}

// Plain (non-TMA) staging of a float tile into the padded layout.
template <int A>
__device__ void load_tile_plain(float* v, const float* __restrict__ x, const FieldGeo& g, const TileInfo& ti)
{
    using TG = TileGeom<A>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rows = (ti.e[0] + 1) * (ti.e[1] + 1);
    for (int rr = warp; rr < rows; rr += nw) {
        const int c0 = rr / (ti.e[1] + 1);
        const int c1 = rr - c0 * (ti.e[1] + 1);
        const float* src = x + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2];
        for (int c2 = lane; c2 <= ti.e[2]; c2 += 32) v[c0 * TG::PY + c1 * TG::PX + c2] = src[c2];
    }
}

template <int A>
__device__ void load_codes_plain(uint8_t* cs, const uint8_t* __restrict__ codes, const FieldGeo& g,
                                 const TileInfo& ti)
{
    using TG = TileGeom<A>;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int rows = (ti.e[0] + 1) * (ti.e[1] + 1);
    for (int rr = warp; rr < rows; rr += nw) {
        const int c0 = rr / (ti.e[1] + 1);
        const int c1 = rr - c0 * (ti.e[1] + 1);
        const uint8_t* src = codes + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2];
        for (int c2 = lane; c2 <= ti.e[2]; c2 += 32) cs[c0 * TG::CY + c1 * TG::CX + c2] = src[c2];
    }
}

// Stage one tile with TMA (one elected thread issues, everybody waits on the
// mbarrier phase).  Returns false, CTA-uniformly, if the bounded wait ran out.
__device__ __forceinline__ bool tma_stage(void* dst, const CUtensorMap* map, const int o[3], uint64_t* mbar,
                                          uint32_t bytes, uint32_t& phase)
{
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(mbar, bytes);
        tma_load_3d(dst, map, o[2], o[1], o[0], mbar);
    }
    const bool ok = mbar_wait(mbar, phase, kSpinLimit);
    phase ^= 1u;
    return __syncthreads_and(ok) != 0;
}

// ---------------------------------------------------------------------------
// Predict + quantize
// ---------------------------------------------------------------------------
template <int A>
__global__ void __launch_bounds__(256) k_compress(const __grid_constant__ CUtensorMap tmap, const FieldGeo g,
                                                  const float* __restrict__ x, uint8_t* __restrict__ codes,
                                                  float* __restrict__ anchors, uint32_t* __restrict__ out_idx,
                                                  float* __restrict__ out_val, const uint64_t out_cap,
                                                  uint32_t* __restrict__ hist_g, float* __restrict__ recon_g,
                                                  hi_header* __restrict__ hdr, const uint32_t tma_bytes,
                                                  const int flags)
{
    using TG = TileGeom<A>;
    extern __shared__ __align__(128) unsigned char smem[];
    float* v = reinterpret_cast<float*>(smem);
    uint8_t* cs = smem + ((g.b0 * TG::P * TG::PX * 4 + 127) / 128) * 128;
    __shared__ uint32_t s_hist[256];
    __shared__ uint16_t s_out[kOutCap];
    __shared__ int s_nout;
    __shared__ unsigned long long s_obase;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ hi_level s_lv[HI_MAX_LEVELS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool use_tma = flags & kFlagTma;
    {   // an earlier stage failed (bad range, device-side EINVAL): leave outputs untouched
        const uint32_t st = hdr->status;
        if (__syncthreads_or(st != 0 && st != HI_ECAPACITY)) return;
    }
    const float eb_f = hdr->eb_f, ebx2_f = hdr->ebx2_f, r_f = hdr->r_f;

    for (int i = tid; i < 256; i += blockDim.x) s_hist[i] = 0;
    if (tid < HI_MAX_LEVELS) s_lv[tid] = hdr->level[tid];
    if (tid == 0) {
        mbar_init(&s_mbar, 1);
        fence_mbar_init();
        if (use_tma) prefetch_tmap(&tmap);
    }
    __syncthreads();

    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        const TileInfo ti = tile_info<A>(g, tile);
        if (tid == 0) s_nout = 0;
        if (use_tma) {
            if (!tma_stage(v, &tmap, ti.o, &s_mbar, tma_bytes, phase)) {
                if (tid == 0) set_status(&hdr->status, HI_ETIMEOUT);
                mbar_wait(&s_mbar, phase ^ 1u, kSpinLimit);
                return;
            }
        } else {
            load_tile_plain<A>(v, x, g, ti);
            __syncthreads();
        }
        // anchors keep the zero-error code
        if (tid < 8) {
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            if (a0 * A <= ti.e[0] && a1 * A <= ti.e[1] && a2 * A <= ti.e[2])
                cs[a0 * A * TG::CY + a1 * A * TG::CX + a2 * A] = (uint8_t)kRadius;
        }

        for (int l = TG::L - 1; l >= 0; --l) {
            const hi_level lv = s_lv[l];
            const bool cubic = lv.interp == HI_CUBIC;
            const int s = 1 << l;
            for (int p = 0; p < 3; ++p) {
                const PassGeom pg = pass_geom(lv, p, s, ti.e);
                if (pg.nd == 0) continue;  // CTA-uniform
                const int ed = pick3(ti.e, pg.d);
                const int vpd = vpitch<A>(pg.d) * s, cpd = cpitch<A>(pg.d) * s;
                const int nlines = pg.nq * pg.nr;
                for (int l0 = warp * 32; l0 < nlines; l0 += blockDim.x) {
                    const int line = l0 + lane;
                    const bool act = line < nlines;
                    const int jq = act ? line / pg.nr : 0;
                    const int jr = act ? line - jq * pg.nr : 0;
                    const int cq = jq * pg.stq, cr = jr * pg.str;
                    const int vb = cq * vpitch<A>(pg.q) + cr * vpitch<A>(pg.r);
                    const int cb = cq * cpitch<A>(pg.q) + cr * cpitch<A>(pg.r);
                    const bool lown = act && cq <= pick3(ti.own, pg.q) && cr <= pick3(ti.own, pg.r);
                    const int ownd = pick3(ti.own, pg.d);
                    float fa = 0.0f, fb = v[vb];
                    float fu = (2 * s <= ed) ? v[vb + 2 * vpd] : 0.0f;
                    float fv = (4 * s <= ed) ? v[vb + 4 * vpd] : 0.0f;
                    for (int k = 0; k < pg.nd; ++k) {
                        const int c = (2 * k + 1) * s;
                        const bool have_r = c + s <= ed, have_l3 = k >= 1, have_r3 = c + 3 * s <= ed;
                        const float pr = predict(cubic, have_l3, have_r, have_r3, fa, fb, fu, fv);
                        const int vi = vb + (2 * k + 1) * vpd;
                        const float xv = v[vi];
                        float xr;
                        const int code = quantize(xv, pr, eb_f, ebx2_f, r_f, xr);
                        if (act) {
                            v[vi] = xr;
                            cs[cb + (2 * k + 1) * cpd] = (uint8_t)code;
                        }
                        if (code == 0 && lown && c <= ownd) {
                            const int slot = atomicAdd(&s_nout, 1);
                            if (slot < kOutCap) {
                                s_out[slot] = (uint16_t)vi;
                            } else {  // overflow: write through directly
                                const unsigned long long pos = atomicAdd(
                                    reinterpret_cast<unsigned long long*>(&hdr->n_outliers), 1ull);
                                if (pos < out_cap) {
                                    out_idx[pos] = (uint32_t)global_index<A>(g, ti.o, vi);
                                    out_val[pos] = xv;
                                } else {
                                    set_status(&hdr->status, HI_ECAPACITY);
                                }
                            }
                        }
                        fa = fb;
                        fb = fu;
                        fu = fv;
                        fv = ((2 * k + 6) * s <= ed) ? v[vb + (2 * k + 6) * vpd] : 0.0f;
                    }
                }
                __syncthreads();
            }
        }

        // ---- epilogue: owned codes (+ histogram), recon, anchors, outliers
        const int own0 = ti.own[0] + 1, own1 = ti.own[1] + 1, own2 = ti.own[2] + 1;
        const int rows = own0 * own1;
        const bool vec_codes = (flags & kFlagVecCodes) && own2 == A && A >= 8;
        if constexpr (A < 8) {
            (void)vec_codes;
        } else if (vec_codes) {
            constexpr int CH = (A >= 16) ? 16 : 8;  // bytes per chunk
            constexpr int NCH = A / CH;
            const int items = rows * NCH;
            for (int i0 = 0; i0 < items; i0 += blockDim.x) {
                const int i = i0 + tid;
                const bool act = i < items;
                const int row = act ? i / NCH : 0, ch = act ? i - row * NCH : 0;
                const int c0 = row / own1, c1 = row - c0 * own1;
                const uint8_t* src = cs + c0 * TG::CY + c1 * TG::CX + ch * CH;
                uint8_t* dst = codes + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] +
                               ch * CH;
                uint32_t w[4];
                if (CH == 16) {
                    const uint4 q4 = *reinterpret_cast<const uint4*>(src);
                    w[0] = q4.x, w[1] = q4.y, w[2] = q4.z, w[3] = q4.w;
                    if (act) *reinterpret_cast<uint4*>(dst) = q4;
                } else {
                    const uint2 q2 = *reinterpret_cast<const uint2*>(src);
                    w[0] = q2.x, w[1] = q2.y, w[2] = 0, w[3] = 0;
                    if (act) *reinterpret_cast<uint2*>(dst) = q2;
                }
                if (hist_g) {
#pragma unroll
                    for (int b = 0; b < CH; ++b) hist_add(s_hist, (w[b >> 2] >> (8 * (b & 3))) & 0xff, act, lane);
                }
            }
        }
        if (!(A >= 8 && vec_codes)) {
            const int items = rows * own2;
            for (int i0 = 0; i0 < items; i0 += blockDim.x) {
                const int i = i0 + tid;
                const bool act = i < items;
                const int row = act ? i / own2 : 0, c2 = act ? i - row * own2 : 0;
                const int c0 = row / own1, c1 = row - c0 * own1;
                const int code = cs[c0 * TG::CY + c1 * TG::CX + c2];
                if (act)
                    codes[((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2] =
                        (uint8_t)code;
                if (hist_g) hist_add(s_hist, code, act, lane);
            }
        }
        if (recon_g) {
            const int items = rows * own2;
            for (int i = tid; i < items; i += blockDim.x) {
                const int row = i / own2, c2 = i - row * own2;
                const int c0 = row / own1, c1 = row - c0 * own1;
                recon_g[((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2] =
                    v[c0 * TG::PY + c1 * TG::PX + c2];
            }
        }
        if (tid < 8) {  // owned anchors, verbatim (Sec. 3.2)
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            const int l0 = a0 * A, l1 = a1 * A, l2 = a2 * A;
            if (l0 <= ti.own[0] && l1 <= ti.own[1] && l2 <= ti.own[2]) {
                const int64_t ai = ((int64_t)(ti.o[0] / A + a0) * g.na[1] + (ti.o[1] / A + a1)) * g.na[2] +
                                   (ti.o[2] / A + a2);
                anchors[ai] = v[l0 * TG::PY + l1 * TG::PX + l2];
                if (hist_g) atomicSub(&s_hist[kRadius], 1u);  // anchors are not predicted
            }
        }
        __syncthreads();
        const int nout = s_nout < kOutCap ? s_nout : kOutCap;
        if (nout > 0) {  // CTA-uniform
            if (tid == 0)
                s_obase = atomicAdd(reinterpret_cast<unsigned long long*>(&hdr->n_outliers),
                                    (unsigned long long)nout);
            __syncthreads();
            for (int i = tid; i < nout; i += blockDim.x) {
                const unsigned long long pos = s_obase + i;
                const int vi = s_out[i];
                if (pos < out_cap) {
                    out_idx[pos] = (uint32_t)global_index<A>(g, ti.o, vi);
                    out_val[pos] = v[vi];
                } else if (i == 0 || pos == out_cap) {
                    set_status(&hdr->status, HI_ECAPACITY);
                }
            }
        }
        // keep the buffers until every thread is done; order the generic-proxy
        // writes above before the next TMA overwrite
        fence_proxy_async_smem();
        __syncthreads();
    }
    if (hist_g) {
        for (int i = tid; i < 256; i += blockDim.x)
            if (s_hist[i]) atomicAdd(&hist_g[i], s_hist[i]);
    }
}

// ---------------------------------------------------------------------------
// Reconstruct
// ---------------------------------------------------------------------------
template <int A>
__global__ void __launch_bounds__(256) k_decompress(const __grid_constant__ CUtensorMap cmap, const FieldGeo g,
                                                    const uint8_t* __restrict__ codes,
                                                    const float* __restrict__ anchors, float* out,
                                                    const hi_header* __restrict__ hdr,
                                                    uint32_t* __restrict__ status, const uint32_t tma_bytes,
                                                    const int flags)
{
    using TG = TileGeom<A>;
    extern __shared__ __align__(128) unsigned char smem[];
    float* v = reinterpret_cast<float*>(smem);
    uint8_t* cs = smem + ((g.b0 * TG::P * TG::PX * 4 + 127) / 128) * 128;
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ hi_level s_lv[HI_MAX_LEVELS];

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const bool use_tma = flags & kFlagTma;
    if (__syncthreads_or(status != nullptr && *status != 0)) return;
    const float ebx2_f = hdr->ebx2_f;
    if (tid < HI_MAX_LEVELS) s_lv[tid] = hdr->level[tid];
    if (tid == 0) {
        mbar_init(&s_mbar, 1);
        fence_mbar_init();
        if (use_tma) prefetch_tmap(&cmap);
    }
    __syncthreads();

    uint32_t phase = 0;
    for (int tile = blockIdx.x; tile < g.ntiles; tile += gridDim.x) {
        const TileInfo ti = tile_info<A>(g, tile);
        if (tid < 8) {  // seed the anchors
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            const int l0 = a0 * A, l1 = a1 * A, l2 = a2 * A;
            if (l0 <= ti.e[0] && l1 <= ti.e[1] && l2 <= ti.e[2]) {
                const int64_t ai = ((int64_t)(ti.o[0] / A + a0) * g.na[1] + (ti.o[1] / A + a1)) * g.na[2] +
                                   (ti.o[2] / A + a2);
                v[l0 * TG::PY + l1 * TG::PX + l2] = anchors[ai];
            }
        }
        if (use_tma) {
            if (!tma_stage(cs, &cmap, ti.o, &s_mbar, tma_bytes, phase)) {
                if (tid == 0) set_status(status, HI_ETIMEOUT);
                mbar_wait(&s_mbar, phase ^ 1u, kSpinLimit);
                return;
            }
        } else {
            load_codes_plain<A>(cs, codes, g, ti);
            __syncthreads();
        }

        for (int l = TG::L - 1; l >= 0; --l) {
            const hi_level lv = s_lv[l];
            const bool cubic = lv.interp == HI_CUBIC;
            const int s = 1 << l;
            for (int p = 0; p < 3; ++p) {
                const PassGeom pg = pass_geom(lv, p, s, ti.e);
                if (pg.nd == 0) continue;
                const int ed = pick3(ti.e, pg.d);
                const int vpd = vpitch<A>(pg.d) * s, cpd = cpitch<A>(pg.d) * s;
                const int nlines = pg.nq * pg.nr;
                for (int l0 = warp * 32; l0 < nlines; l0 += blockDim.x) {
                    const int line = l0 + lane;
                    const bool act = line < nlines;
                    const int jq = act ? line / pg.nr : 0;
                    const int jr = act ? line - jq * pg.nr : 0;
                    const int cq = jq * pg.stq, cr = jr * pg.str;
                    const int vb = cq * vpitch<A>(pg.q) + cr * vpitch<A>(pg.r);
                    const int cb = cq * cpitch<A>(pg.q) + cr * cpitch<A>(pg.r);
                    float fa = 0.0f, fb = v[vb];
                    float fu = (2 * s <= ed) ? v[vb + 2 * vpd] : 0.0f;
                    float fv = (4 * s <= ed) ? v[vb + 4 * vpd] : 0.0f;
                    for (int k = 0; k < pg.nd; ++k) {
                        const int c = (2 * k + 1) * s;
                        const bool have_r = c + s <= ed, have_l3 = k >= 1, have_r3 = c + 3 * s <= ed;
                        const float pr = predict(cubic, have_l3, have_r, have_r3, fa, fb, fu, fv);
                        const int vi = vb + (2 * k + 1) * vpd;
                        const int code = cs[cb + (2 * k + 1) * cpd];
                        float xr = dequantize(code, pr, ebx2_f);
                        if (code == 0 && act) xr = out[global_index<A>(g, ti.o, vi)];
                        if (act) v[vi] = xr;
                        fa = fb;
                        fb = fu;
                        fu = fv;
                        fv = ((2 * k + 6) * s <= ed) ? v[vb + (2 * k + 6) * vpd] : 0.0f;
                    }
                }
                __syncthreads();
            }
        }

        // ---- epilogue: owned reconstructed values
        const int own0 = ti.own[0] + 1, own1 = ti.own[1] + 1, own2 = ti.own[2] + 1;
        const int rows = own0 * own1;
        const bool vec_out = (flags & kFlagVecOut) && own2 == A && A >= 4;
        if constexpr (A < 4) {
            (void)vec_out;
        } else if (vec_out) {
            constexpr int NCH = A / 4;
            const int items = rows * NCH;
            for (int i = tid; i < items; i += blockDim.x) {
                const int row = i / NCH, ch = i - row * NCH;
                const int c0 = row / own1, c1 = row - c0 * own1;
                const float4 f4 = *reinterpret_cast<const float4*>(v + c0 * TG::PY + c1 * TG::PX + ch * 4);
                *reinterpret_cast<float4*>(out + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] +
                                           ti.o[2] + ch * 4) = f4;
            }
        }
        if (!(A >= 4 && vec_out)) {
            const int items = rows * own2;
            for (int i = tid; i < items; i += blockDim.x) {
                const int row = i / own2, c2 = i - row * own2;
                const int c0 = row / own1, c1 = row - c0 * own1;
                out[((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2] =
                    v[c0 * TG::PY + c1 * TG::PX + c2];
            }
        }
        fence_proxy_async_smem();
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------
template <int A>
size_t tile_smem_bytes(int b0)
{
    using TG = TileGeom<A>;
    const size_t vb = ((size_t)b0 * TG::P * TG::PX * 4 + 127) / 128 * 128;
    return vb + (size_t)b0 * TG::P * TG::CX;
}

template <int A>
static cudaError_t launch_compress_t(const CompressLaunch& c, cudaStream_t st)
{
    const size_t smem = tile_smem_bytes<A>(c.g.b0);
    auto kern = k_compress<A>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, c.threads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    int grid = per_sm * c.num_sms;
    if (grid > c.g.ntiles) grid = c.g.ntiles;
    if (c.max_ctas > 0 && grid > c.max_ctas) grid = c.max_ctas;
    kern<<<grid, c.threads, smem, st>>>(c.tmap, c.g, c.x, c.codes, c.anchors, c.out_idx, c.out_val, c.out_cap,
                                        c.hist, c.recon, c.hdr, c.tma_bytes, c.flags);
    return cudaGetLastError();
}

template <int A>
static cudaError_t launch_decompress_t(const DecompressLaunch& c, cudaStream_t st)
{
    const size_t smem = tile_smem_bytes<A>(c.g.b0);
    auto kern = k_decompress<A>;
    cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, c.threads, smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    int grid = per_sm * c.num_sms;
    if (grid > c.g.ntiles) grid = c.g.ntiles;
    if (c.max_ctas > 0 && grid > c.max_ctas) grid = c.max_ctas;
    kern<<<grid, c.threads, smem, st>>>(c.cmap, c.g, c.codes, c.anchors, c.out, c.hdr, c.status, c.tma_bytes,
                                        c.flags);
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
    case 2: return tile_smem_bytes<2>(b0);
    case 4: return tile_smem_bytes<4>(b0);
    case 8: return tile_smem_bytes<8>(b0);
    case 16: return tile_smem_bytes<16>(b0);
    case 32: return tile_smem_bytes<32>(b0);
    default: return 0;
    }
}

}  // namespace hi
