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

// The level passes of one staged tile (codes in cs, anchors seeded in v).
template <int A>
__device__ __forceinline__ void decompress_levels(const TileInfo& ti, float* v, const uint8_t* cs, const int* s_sel,
                                                  const hi_level* s_lv, const Hot h, bool full_ok)
{
    uint8_t* csw = const_cast<uint8_t*>(cs);
    const bool full = full_ok && ti.e[0] == A && ti.e[1] == A && ti.e[2] == A;
    if constexpr (HasFull<A>::value) {
        if (full)
            levels_full<A, TileGeom<A>::L - 1, false>(s_sel, v, csw, h);
        else
            levels_ragged<A, TileGeom<A>::L - 1, false>(s_lv, v, csw, h, ti);
    } else {
        levels_ragged<A, TileGeom<A>::L - 1, false>(s_lv, v, csw, h, ti);
    }
}

// The owned reconstructed values of a tile to the output field.
template <int A>
__device__ __forceinline__ void decompress_store(const FieldGeo& g, const TileInfo& ti, const float* v, float* out,
                                                 bool vec_ok)
{
    using Lw = Lay<A>;
    const int tid = threadIdx.x;
    const int own0 = ti.own[0] + 1, own1 = ti.own[1] + 1, own2 = ti.own[2] + 1;
    const int rows = own0 * own1;
    const bool vec_out = vec_ok && own2 == A && A >= 4;
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
        decompress_levels<A>(ti, v, cs, s_sel, s_lv, h, full_ok);

        if constexpr (EARLY) {  // launched only with TMA staging and one buffer
            // order the passes' generic reads of cs before the copy that overwrites it
            fence_proxy_async_smem();
            __syncthreads();
            if (tid == 0 && next < g.ntiles) tma_issue(cs, &cmap, g, shell_first(g, next), A, &s_mbar[0], tma_bytes);
        }

        decompress_store<A>(g, ti, v, out, (flags & kFlagVecOut) != 0);
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

// ---------------------------------------------------------------------------
// Batched reconstruction: every field of a prepared batch, two launches
// ---------------------------------------------------------------------------
// A field is reconstructed when its header is a valid record without an
// error and its outliers fit the capacity of its arrays.
__device__ __forceinline__ bool batch_field_ok(const BatchField& F)
{
    const hi_header* hdr = F.hdr;
    return hdr->magic == HI_MAGIC && hdr->status == 0 && hdr->n_outliers <= F.out_cap;
}

// Outlier values of every field into its output (blockIdx.y = field); block
// (0, 0) also zeroes the reconstruction queue.
__global__ void __launch_bounds__(256) k_batch_scatter(const BatchField* __restrict__ fields,
                                                       uint32_t* __restrict__ status, uint32_t* __restrict__ queue)
{
    const BatchField& F = fields[blockIdx.y];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) *queue = 0;
    if (!batch_field_ok(F)) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const hi_header* hdr = F.hdr;
            const bool cap = hdr->magic == HI_MAGIC && (hdr->status == HI_ECAPACITY || hdr->n_outliers > F.out_cap);
            set_status(status, cap ? HI_ECAPACITY : HI_ECORRUPT);
        }
        return;
    }
    const uint64_t n = F.hdr->n_outliers;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k = F.out_idx[i];
        if ((int64_t)k < F.g.N)
            F.out[k] = F.out_val[i];
        else
            set_status(status, HI_ECORRUPT);
    }
}

// Persistent over the (field, tile) work items of all fields, whole 3D tiles
// of every field first: a code tile staged by TMA (or plain loads), the
// field's corner anchors seeded, the level passes under the field's
// configuration (from its header, reloaded when the field changes), the
// owned values to the field's output.  One tile buffer.
template <int A>
__global__ void __launch_bounds__(kMaxThreads, 6)
    k_decompress_batch(const BatchField* __restrict__ fields, const uint32_t* __restrict__ head_start,
                       const uint32_t* __restrict__ shell_start, const int n, const uint32_t total_head,
                       const uint32_t total, uint32_t* __restrict__ queue, uint32_t* __restrict__ status)
{
    using Lw = Lay<A>;
    extern __shared__ __align__(128) unsigned char smem[];
    float* const v = reinterpret_cast<float*>(smem);
    uint8_t* const cs = smem + vbuf_bytes<A>(A + 1);
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ hi_level s_lv[HI_MAX_LEVELS];
    __shared__ int s_sel[HI_MAX_LEVELS];
    __shared__ int s_next, s_skip;
    __shared__ int s_tf[2];
    __shared__ TileInfo s_ti[2];
    __shared__ float s_ebx2;
    const int tid = threadIdx.x;
    if (tid == 0) {
        mbar_init(&s_mbar, 1);
        fence_mbar_init();
        if (blockIdx.x < total) {
            int pos;
            const int f = batch_locate(fields, head_start, shell_start, n, total_head, blockIdx.x, &pos);
            s_tf[0] = f;
            s_ti[0] = tile_info<A>(fields[f].g, pos);
        }
    }
    __syncthreads();
    int cur = -1;
    uint32_t ph = 0;
    int it = 0;
    for (uint32_t w = blockIdx.x; w < total; ++it) {
        const int f = s_tf[it & 1];
        const TileInfo ti = s_ti[it & 1];
        const BatchField& F = fields[f];
        if (f != cur) {  // a new field: its level configuration and constants
            if (tid < HI_MAX_LEVELS) {
                s_lv[tid] = F.hdr->level[tid];
                s_sel[tid] = perm_sel(s_lv[tid]);
            }
            if (tid == 0) {
                s_ebx2 = F.hdr->ebx2_f;
                s_skip = batch_field_ok(F) ? 0 : 1;
            }
            __syncthreads();
            cur = f;
        }
        const bool tma = (F.dflags & kFlagTma) != 0;
        if (tid == 0) {
            s_rare.out = F.out;
            s_rare.g = F.g;
            s_rare.o[0] = ti.o[0], s_rare.o[1] = ti.o[1], s_rare.o[2] = ti.o[2];
            if (tma) {  // the buffer is free again (the last iteration's closing barrier)
                mbar_arrive_expect_tx(&s_mbar, F.ctma_bytes);
                tma_load_3d(cs, &F.cmap, ti.o[2], ti.o[1], ti.o[0], &s_mbar);
            }
            const uint32_t nx = gridDim.x + atomicAdd(queue, 1u);
            s_next = (int)(nx < total ? nx : total);
            if (nx < total) {
                int pos;
                const int fn = batch_locate(fields, head_start, shell_start, n, total_head, nx, &pos);
                s_tf[(it + 1) & 1] = fn;
                s_ti[(it + 1) & 1] = tile_info<A>(fields[fn].g, pos);
            }
        }
        if (tid < 8) {  // seed the corner anchors
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            const int l0 = a0 * A, l1 = a1 * A, l2 = a2 * A;
            if (l0 <= ti.e[0] && l1 <= ti.e[1] && l2 <= ti.e[2]) {
                const FieldGeo& g = F.g;
                v[l0 * Lw::PY + l1 * Lw::PX + l2] =
                    F.anchors[((int64_t)(ti.o[0] / A + a0) * g.na[1] + (ti.o[1] / A + a1)) * g.na[2] + (ti.o[2] / A + a2)];
            }
        }
        if (tma) {
            const bool ok = mbar_wait(&s_mbar, ph, kSpinLimit);
            ph ^= 1u;
            if (!__syncthreads_and(ok)) {
                // the copy this CTA issued may still be in flight: stay until it lands
                if (tid == 0) set_status(status, HI_ETIMEOUT);
                drain_wait(&s_mbar, ph ^ 1u);
                __syncthreads();
                return;
            }
        } else {
            load_codes_plain<A>(cs, F.codes, F.g, ti);
            __syncthreads();
        }
        const int next = s_next;
        if (!s_skip) {
            Hot h;
            h.eb_f = 0.0f;
            h.ebx2_f = s_ebx2;
            h.r_f = 0.0f;
            const bool full_ok = HasFull<A>::value && F.g.n[0] > 1 && F.g.n[1] > 1 && F.g.n[2] > 1;
            decompress_levels<A>(ti, v, cs, s_sel, s_lv, h, full_ok);
            decompress_store<A>(F.g, ti, v, F.out, (F.dflags & kFlagVecOut) != 0);
        }
        // keep the buffers until every thread is done; order the generic-proxy
        // reads above before the next TMA write of the code buffer
        fence_proxy_async_smem();
        __syncthreads();
        w = (uint32_t)next;
    }
}

cudaError_t launch_batch_scatter(const BatchLaunch& b, uint32_t* status, uint32_t* queue, cudaStream_t st)
{
    k_batch_scatter<<<dim3(64, (unsigned)b.n), 256, 0, st>>>(b.fields, status, queue);
    return cudaGetLastError();
}

template <int A>
static cudaError_t launch_decompress_batch_t(const BatchLaunch& b, uint32_t* status, uint32_t* queue, cudaStream_t st)
{
    auto kern = k_decompress_batch<A>;
    const size_t smem = decompress_smem_t<A>(A + 1, false);
    int grid = 0;
    cudaError_t err = persistent_grid(kern, kMaxThreads, smem, b.num_sms, (int)b.total_tiles, 0, &grid);
    if (err != cudaSuccess) return err;
    kern<<<grid, kMaxThreads, smem, st>>>(b.fields, b.tile_start, b.shell_start, b.n, b.total_head, b.total_tiles,
                                          queue, status);
    return cudaGetLastError();
}

cudaError_t launch_decompress_batch(const BatchLaunch& b, uint32_t* status, uint32_t* queue, cudaStream_t st)
{
    switch (b.A) {
    case 8: return launch_decompress_batch_t<8>(b, status, queue, st);
    case 16: return launch_decompress_batch_t<16>(b, status, queue, st);
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

}  // namespace hi
