// hi_batch.cu -- many fields of uneven shapes compressed together: one launch
// per stage for the whole batch (header set-up, value range, auto-tune,
// predict + quantize).  The predict + quantize kernel is persistent: its CTAs
// take (field, tile) work items from one queue over the concatenated tile
// lists of all fields, so small and large fields share the GPU without a
// launch per field.  Each field's results are those of a single-field
// compression of it (Sec. 3.2, Sec. 5.1, Sec. 5.2.1).
#include "hi_aux_dev.cuh"
#include "hi_compress_tile.cuh"

namespace hi {

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

__global__ void k_batch_prologue(const BatchField* __restrict__ fields, uint32_t* queue)
{
    const BatchField& F = fields[blockIdx.x];
    prologue_fill(F.hdr, F.p, F.n_anchors, F.out_cap, F.n_levels, F.hist, F.tickets, F.tickets + 1,
                  blockIdx.x == 0 ? queue : nullptr);
}

// Value range of every relative-bound field: work item = kBatchChunk points
// of one field; the last item of a field to finish folds its partials.
__global__ void __launch_bounds__(512) k_batch_range(const BatchField* __restrict__ fields,
                                                     const uint32_t* __restrict__ chunk_start, int n, uint32_t total)
{
    __shared__ float s_mn[32], s_mx[32];
    __shared__ bool s_last;
    for (uint32_t c = blockIdx.x; c < total; c += gridDim.x) {
        const int f = find_field(chunk_start, n, c);
        const BatchField& F = fields[f];
        const uint32_t k = c - __ldg(chunk_start + f);
        const int64_t lo = (int64_t)k * kBatchChunk;
        const int64_t hi = (lo + kBatchChunk < F.g.N) ? lo + kBatchChunk : F.g.N;
        float mn = INFINITY, mx = -INFINITY;
        range_accum(F.x, lo, hi, threadIdx.x, blockDim.x, mn, mx);
        block_minmax(mn, mx, s_mn, s_mx);
        if (threadIdx.x == 0) {
            F.partials[k] = make_float2(mn, mx);
            __threadfence();
            s_last = atomicAdd(&F.tickets[0], 1u) == F.nchunks - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            range_fold(F.partials, F.nchunks, F.hdr, s_mn, s_mx);
            if (threadIdx.x == 0) F.tickets[0] = 0;
        }
        __syncthreads();
    }
}

// Auto-tune of every field that asks for it: blockIdx.x = a sample of some
// field, blockIdx.y = candidate (beyond the field's count: nothing to do).
template <int A>
__global__ void __launch_bounds__(256) k_batch_tune(const BatchField* __restrict__ fields,
                                                    const uint32_t* __restrict__ sample_start, int n)
{
    extern __shared__ __align__(128) unsigned char smem[];
    const int f = find_field(sample_start, n, blockIdx.x);
    const BatchField& F = fields[f];
    if ((int)blockIdx.y >= F.cands.ncfg) return;
    if (F.hdr->status != 0) return;  // the range stage failed: keep the given levels
    tune_block<A>(reinterpret_cast<float*>(smem), &F.tmap, F.g, F.x, F.cands, blockIdx.x - __ldg(sample_start + f),
                  blockIdx.y, F.stride, F.m, F.err, &F.tickets[1], F.hdr, F.tma_bytes, (F.flags & kFlagTma) != 0);
}

// Thread 0 of a batched CTA, at the top of iteration `it` on work item
// (f, lt) staged in v: takes the next work item from the queue, decodes its
// field and tile into slot (it + 1) & 1, and starts the copies: with two
// buffers the next tile's box into `other`; with one, this tile's box (the
// buffer is free again) and an L2 prefetch of the next one.
template <int A>
__device__ __forceinline__ void batch_schedule(const BatchField* __restrict__ fields,
                                            const uint32_t* __restrict__ tile_start, int n, uint32_t total,
                                            uint32_t* queue, int it, bool dbuf, int f, int lt, bool tma_here,
                                            float* v, float* other, uint64_t* s_mbar, int* s_next, int* s_tf,
                                            int* s_tl, int* s_tma, TileInfo* s_ti)
{
    const int buf = dbuf ? (it & 1) : 0;
    const uint32_t nx = gridDim.x + atomicAdd(queue, 1u);
    *s_next = (int)(nx < total ? nx : total);
    int fn = -1, ln = 0;
    if (nx < total) {
        fn = find_field(tile_start, n, nx);
        ln = (int)(nx - __ldg(tile_start + fn));
        s_tf[(it + 1) & 1] = fn;
        s_tl[(it + 1) & 1] = ln;
        s_ti[(it + 1) & 1] = tile_info<A>(fields[fn].g, ln);
        s_tma[(it + 1) & 1] = (fields[fn].flags & kFlagTma) != 0;
    }
    if (dbuf && fn >= 0 && (fields[fn].flags & kFlagTma))
        tma_issue(other, &fields[fn].tmap, fields[fn].g, ln, A, &s_mbar[buf ^ 1], fields[fn].tma_bytes);
    if (!dbuf && it > 0 && tma_here) tma_issue(v, &fields[f].tmap, fields[f].g, lt, A, &s_mbar[0], fields[f].tma_bytes);
    if (!dbuf && fn >= 0 && (fields[fn].flags & kFlagTma)) tma_l2_prefetch(&fields[fn].tmap, fields[fn].g, ln, A);
}

// Per-field state of the field a CTA is working on (shared memory).
struct BatchCur {
    CompressOut out;
    FieldGeo g;
    const float* x;
    uint32_t* hist;
    Hot h;
    int flags;
    int skip;     // an earlier stage of this field failed: leave its outputs
    int full_ok;  // every dim active: whole tiles take the compile-time passes
};

template <int A>
__global__ void __launch_bounds__(kMaxThreads, 5)
    k_compress_batch(const BatchField* __restrict__ fields, const uint32_t* __restrict__ tile_start, const int n,
                     const uint32_t total, uint32_t* __restrict__ queue, const int dbuf_flag)
{
    using Lw = Lay<A>;
    extern __shared__ __align__(128) unsigned char smem[];
    const bool dbuf = dbuf_flag != 0;
    const int vb_bytes = vbuf_bytes<A>(A + 1);
    float* const vbuf0 = reinterpret_cast<float*>(smem);
    float* const vbuf1 = reinterpret_cast<float*>(smem + (dbuf ? vb_bytes : 0));
    uint8_t* cs = smem + (dbuf ? 2 : 1) * vb_bytes;
    uint16_t* hc = reinterpret_cast<uint16_t*>(cs + round128((A + 1) * Lw::P * Lw::CXC));
    __shared__ uint32_t s_hist[256];
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ hi_level s_lv[HI_MAX_LEVELS];
    __shared__ int s_sel[HI_MAX_LEVELS];
    __shared__ BatchCur s_cur;
    __shared__ int s_next;
    __shared__ int s_tf[2];    // field of this work item and of the next
    __shared__ int s_tl[2];    // its tile within the field (queue order)
    __shared__ int s_tma[2];   // staged by TMA
    __shared__ TileInfo s_ti[2];

    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += blockDim.x) s_hist[i] = 0;
    for (int k = 0; k < kHistBins; ++k) hc[k * blockDim.x + tid] = 0;
    if (tid == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        fence_mbar_init();
        if (blockIdx.x < total) {
            const int f = find_field(tile_start, n, blockIdx.x);
            const BatchField& F = fields[f];
            const int lt = (int)(blockIdx.x - __ldg(tile_start + f));
            s_tf[0] = f;
            s_tl[0] = lt;
            s_ti[0] = tile_info<A>(F.g, lt);
            s_tma[0] = (F.flags & kFlagTma) != 0;
            if (s_tma[0]) tma_issue(vbuf0, &F.tmap, F.g, lt, A, &s_mbar[0], F.tma_bytes);
        }
    }
    __syncthreads();

    int cur = -1;
    uint32_t ph = 0;  // bit b: phase of buffer b's barrier
    int it = 0;
    for (uint32_t w = blockIdx.x; w < total; ++it) {
        const int buf = dbuf ? (it & 1) : 0;
        float* v = buf ? vbuf1 : vbuf0;
        const int f = s_tf[it & 1];
        const int lt = s_tl[it & 1];
        const bool tma_here = s_tma[it & 1] != 0;
        const TileInfo ti = s_ti[it & 1];
        if (tid == 0)
            batch_schedule<A>(fields, tile_start, n, total, queue, it, dbuf, f, lt, tma_here, v, buf ? vbuf0 : vbuf1,
                              s_mbar, &s_next, s_tf, s_tl, s_tma, s_ti);
        if (f != cur) {  // a new field: flush the histogram of the last one, load this one
            if (cur >= 0 && s_cur.hist) hist_flush(hc, s_hist, s_cur.hist);
            __syncthreads();
            if (tid == 0) {
                const BatchField& F = fields[f];
                s_cur.out.codes = F.codes;
                s_cur.out.anchors = F.anchors;
                s_cur.out.out_idx = F.out_idx;
                s_cur.out.out_val = F.out_val;
                s_cur.out.out_cap = F.out_cap;
                s_cur.out.recon = F.recon;
                s_cur.out.hdr = F.hdr;
                s_cur.out.vec_ok = (F.flags & kFlagVecCodes) != 0;
                s_cur.out.hist_on = F.hist != nullptr;
                s_cur.g = F.g;
                s_cur.x = F.x;
                s_cur.hist = F.hist;
                s_cur.h.eb_f = F.hdr->eb_f;
                s_cur.h.ebx2_f = F.hdr->ebx2_f;
                s_cur.h.r_f = F.hdr->r_f;
                s_cur.flags = F.flags;
                const uint32_t st = F.hdr->status;
                s_cur.skip = st != 0 && st != HI_ECAPACITY;
                s_cur.full_ok = HasFull<A>::value && F.g.n[0] > 1 && F.g.n[1] > 1 && F.g.n[2] > 1;
            }
            if (tid < HI_MAX_LEVELS) {
                s_lv[tid] = fields[f].hdr->level[tid];
                s_sel[tid] = perm_sel(s_lv[tid]);
            }
            __syncthreads();
            cur = f;
        }
        if (tid < 8) {  // anchors keep the zero-error code
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            if (a0 * A <= ti.e[0] && a1 * A <= ti.e[1] && a2 * A <= ti.e[2])
                cs[a0 * A * Lw::CYC + a1 * A * Lw::CXC + a2 * A] = (uint8_t)kRadius;
        }
        if (tma_here) {
            const bool ok = mbar_wait(&s_mbar[buf], (ph >> buf) & 1u, kSpinLimit);
            ph ^= 1u << buf;
            if (!__syncthreads_and(ok)) {
                if (tid == 0) set_status(&s_cur.out.hdr->status, HI_ETIMEOUT);
                if (dbuf && s_next < (int)total && s_tma[(it + 1) & 1])
                    mbar_wait(&s_mbar[buf ^ 1], (ph >> (buf ^ 1)) & 1u, kSpinLimit);
                return;
            }
        } else {
            load_tile_plain<A>(v, s_cur.x, s_cur.g, ti);
            __syncthreads();
        }
        const int next = s_next;
        if (!s_cur.skip)
            compress_tile<A>(s_cur.g, ti, v, cs, hc, s_hist, s_sel, s_lv, s_cur.h, s_cur.full_ok != 0, s_cur.out);
        if ((it % kHistFoldTiles) == kHistFoldTiles - 1) hist_fold(hc, s_hist);
        fence_proxy_async_smem();
        __syncthreads();
        w = (uint32_t)next;
    }
    if (cur >= 0 && s_cur.hist) hist_flush(hc, s_hist, s_cur.hist);
}

cudaError_t launch_batch_prologue(const BatchLaunch& b, cudaStream_t st)
{
    k_batch_prologue<<<b.n, 256, 0, st>>>(b.fields, b.queue);
    return cudaGetLastError();
}

cudaError_t launch_batch_range(const BatchLaunch& b, cudaStream_t st)
{
    if (b.total_chunks == 0) return cudaSuccess;
    uint32_t grid = (uint32_t)b.num_sms * 4;
    if (grid > b.total_chunks) grid = b.total_chunks;
    k_batch_range<<<grid, 512, 0, st>>>(b.fields, b.chunk_start, b.n, b.total_chunks);
    return cudaGetLastError();
}

template <int A>
static cudaError_t launch_batch_tune_t(const BatchLaunch& b, cudaStream_t st)
{
    using TG = TileGeom<A>;
    const size_t smem = (size_t)(A + 1) * TG::P * TG::PX * 4;
    auto kern = k_batch_tune<A>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<dim3(b.total_samples, 12), 256, smem, st>>>(b.fields, b.sample_start, b.n);
    return cudaGetLastError();
}

cudaError_t launch_batch_tune(const BatchLaunch& b, cudaStream_t st)
{
    if (b.total_samples == 0) return cudaSuccess;
    switch (b.A) {
    case 8: return launch_batch_tune_t<8>(b, st);
    case 16: return launch_batch_tune_t<16>(b, st);
    default: return cudaErrorInvalidValue;
    }
}

template <int A>
static cudaError_t launch_batch_compress_t(const BatchLaunch& b, cudaStream_t st)
{
    auto kern = k_compress_batch<A>;
    const bool dbuf = b.buffers == 2 && fits_double(kern, compress_smem_t<A>(A + 1, true, b.threads));
    const size_t smem = compress_smem_t<A>(A + 1, dbuf, b.threads);
    int grid = 0;
    cudaError_t err = persistent_grid(kern, b.threads, smem, b.num_sms, (int)b.total_tiles, 0, &grid);
    if (err != cudaSuccess) return err;
    kern<<<grid, b.threads, smem, st>>>(b.fields, b.tile_start, b.n, b.total_tiles, b.queue, dbuf ? 1 : 0);
    return cudaGetLastError();
}

cudaError_t launch_batch_compress(const BatchLaunch& b, cudaStream_t st)
{
    switch (b.A) {
    case 8: return launch_batch_compress_t<8>(b, st);
    case 16: return launch_batch_compress_t<16>(b, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hi
