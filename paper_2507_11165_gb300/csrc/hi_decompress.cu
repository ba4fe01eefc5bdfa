// hi_decompress.cu -- the level-by-level reconstruction (cuSZ-Hi, arXiv
// 2507.11165, Eq. 1, Sec. 3.2): staged code tiles, the level passes
// (hi_passes.cuh) and the epilogue that stores the owned values.
#define HI_LEVEL_FN __noinline__
#include "hi_passes.cuh"

namespace hi {

// ---------------------------------------------------------------------------
// Reconstruct
// ---------------------------------------------------------------------------
// Corner anchor tid (0..7) of the tile at queue position pos, or 0.
template <int A>
__device__ __forceinline__ float anchor_of(const FieldGeo& g, const float* __restrict__ anchors, int pos,
                                           const TileInfo& tn)
{
    const int tid = threadIdx.x;
    if (tid >= 8 || pos >= g.ntiles) return 0.0f;
    const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
    if (a0 * A > tn.e[0] || a1 * A > tn.e[1] || a2 * A > tn.e[2]) return 0.0f;
    return anchors[((int64_t)(tn.o[0] / A + a0) * g.na[1] + (tn.o[1] / A + a1)) * g.na[2] + (tn.o[2] / A + a2)];
}

// Issue a tile's code copy right after the previous tile's passes (one
// buffer): the epilogue only reads the float tile.
constexpr bool kEarlyTmaD = true;

template <int A, bool EARLY>
__global__ void __launch_bounds__(kMaxThreads, 6)
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
    uint8_t* const cbuf0 = smem + vb_bytes;
    uint8_t* const cbuf1 = smem + vb_bytes + (dbuf ? cb_bytes : 0);
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
        if ((int)blockIdx.x < g.ntiles) s_ti[0] = tile_info<A>(g, shell_first(g, blockIdx.x));
        if (use_tma) {
            prefetch_tmap(&cmap);
            if ((int)blockIdx.x < g.ntiles)
                tma_issue(cbuf0, &cmap, g, shell_first(g, blockIdx.x), A, &s_mbar[0], tma_bytes);
        }
    }
    __syncthreads();
    const bool full_ok = HasFull<A>::value && g.n[0] > 1 && g.n[1] > 1 && g.n[2] > 1;

    // the 8 corner anchors of a tile, loaded one tile ahead by threads 0..7
    float a_cur = anchor_of<A>(g, anchors, blockIdx.x, s_ti[0]);

    int it = 0;
    for (int tile = blockIdx.x; tile < g.ntiles; ++it) {
        const int buf = dbuf ? (it & 1) : 0;
        uint8_t* cs = buf ? cbuf1 : cbuf0;
        const TileInfo ti = s_ti[it & 1];
        if (tid == 0) {
            // one buffer: this tile's copy first, before the queue's round trip
            if (use_tma && !dbuf && !EARLY && it > 0)
                tma_issue(cs, &cmap, g, shell_first(g, tile), A, &s_mbar[0], tma_bytes);
            const int nx = (int)gridDim.x + (int)atomicAdd(queue, 1u);
            s_next = nx;
            if (nx < g.ntiles) s_ti[(it + 1) & 1] = tile_info<A>(g, shell_first(g, nx));
            s_rare.o[0] = ti.o[0], s_rare.o[1] = ti.o[1], s_rare.o[2] = ti.o[2];
            if (use_tma && dbuf && nx < g.ntiles)
                tma_issue(buf ? cbuf0 : cbuf1, &cmap, g, shell_first(g, nx), A, &s_mbar[buf ^ 1], tma_bytes);
            // one buffer: the next tile waits in L2 until this one is done
            if (use_tma && !dbuf && nx < g.ntiles) tma_l2_prefetch(&cmap, g, shell_first(g, nx), A);
        }
        if (tid < 8) {  // seed the anchors
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            const int l0 = a0 * A, l1 = a1 * A, l2 = a2 * A;
            if (l0 <= ti.e[0] && l1 <= ti.e[1] && l2 <= ti.e[2]) v[l0 * Lw::PY + l1 * Lw::PX + l2] = a_cur;
        }
        if (use_tma) {
            const bool ok = mbar_wait(&s_mbar[buf], dbuf ? ((it >> 1) & 1) : (it & 1), kSpinLimit);
            if (!__syncthreads_and(ok)) {
                // the copies this CTA issued may still be in flight: record the
                // status and stay until they have landed (or a longer bound ends)
                if (tid == 0) set_status(status, HI_ETIMEOUT);
                drain_wait(&s_mbar[buf], dbuf ? ((it >> 1) & 1) : (it & 1));
                if (dbuf && s_next < g.ntiles) drain_wait(&s_mbar[buf ^ 1], ((it + 1) >> 1) & 1);
                __syncthreads();
                return;
            }
        } else {
            load_codes_plain<A>(cs, codes, g, ti);
            __syncthreads();
            if (s_next < g.ntiles) prefetch_rows_l2<A>(codes, 1, g, s_ti[(it + 1) & 1]);
        }
        const int next = s_next;
        const float a_nxt = anchor_of<A>(g, anchors, next, s_ti[(it + 1) & 1]);  // in flight while this tile is reconstructed
        {
            const bool full = full_ok && ti.e[0] == A && ti.e[1] == A && ti.e[2] == A;
            if constexpr (HasFull<A>::value) {
                if (full)
                    levels_full<A, TileGeom<A>::L - 1, false>(s_sel, v, cs, h);
                else
                    levels_ragged<A, TileGeom<A>::L - 1, false>(s_lv, v, cs, h, ti);
            } else {
                levels_ragged<A, TileGeom<A>::L - 1, false>(s_lv, v, cs, h, ti);
            }
        }

        if constexpr (EARLY) {  // launched only with TMA staging and one buffer
            // order the passes' generic reads of cs before the copy that overwrites it
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0 && next < g.ntiles) tma_issue(cs, &cmap, g, shell_first(g, next), A, &s_mbar[0], tma_bytes);
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
        } else if (own2 <= 32) {
            // lanes over the columns, two rows per warp step when they are at most 16 wide
            const int lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
            const bool two = own2 <= 16;
            const int rpw = two ? 2 : 1;
            const int sub = two ? (lane >> 4) : 0, col = two ? (lane & 15) : lane;
            for (int r0 = warp * rpw; r0 < rows; r0 += nw * rpw) {
                const int row = r0 + sub;
                if (row < rows && col < own2) {
                    const int c0 = row / own1, c1 = row - c0 * own1;
                    out[((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + col] =
                        v[c0 * Lw::PY + c1 * Lw::PX + col];
                }
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

template <int A>
static cudaError_t launch_decompress_t(const DecompressLaunch& c, cudaStream_t st)
{
    const bool dbuf = c.buffers == 2 && fits_double(k_decompress<A, false>, decompress_smem_t<A>(c.g.b0, true));
    const bool early = kEarlyTmaD && (c.flags & kFlagTma) && !dbuf;
    auto kern = early ? k_decompress<A, true> : k_decompress<A, false>;
    const size_t smem = decompress_smem_t<A>(c.g.b0, dbuf);
    int grid = 0;
    cudaError_t err = persistent_grid(kern, c.threads, smem, c.num_sms, c.g.ntiles, c.max_ctas, &grid);
    if (err != cudaSuccess) return err;
    kern<<<grid, c.threads, smem, st>>>(c.cmap, c.g, c.codes, c.anchors, c.out, c.hdr, c.status, c.queue,
                                        c.tma_bytes, c.flags | (dbuf ? kFlagDoubleBuf : 0));
    return cudaGetLastError();
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

}  // namespace hi
