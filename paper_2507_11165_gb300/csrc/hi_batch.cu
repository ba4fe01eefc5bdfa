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

__global__ void k_batch_prologue(const BatchField* __restrict__ fields, uint32_t* queue)
{
    const BatchField& F = fields[blockIdx.x];
    prologue_fill(F.hdr, F.p, F.n_anchors, F.out_cap, F.n_levels, F.hist, F.tickets, F.tickets + 1,
                  blockIdx.x == 0 ? queue : nullptr);
}

// Value range of every relative-bound field: work item = kBatchChunk points
// of one field, items first, first + step, ...; the last item of a field to
// finish folds its partials.
__device__ __forceinline__ void batch_range_items(const BatchField* __restrict__ fields,
                                                  const uint32_t* __restrict__ chunk_start, int n, uint32_t total,
                                                  uint32_t first, uint32_t step)
{
    __shared__ float s_mn[32], s_mx[32];
    __shared__ bool s_last;
    for (uint32_t c = first; c < total; c += step) {
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

// Value range and auto-tune of every field in one launch (neither needs the
// other: the tuner's errors are open-loop, without eps).  Blocks [0, ntune):
// auto-tune, one sample of some field each; the next nb_range blocks: the
// range items.
template <int A>
__global__ void __launch_bounds__(256) k_batch_range_tune(const BatchField* __restrict__ fields,
                                                          const uint32_t* __restrict__ sample_start,
                                                          const uint32_t* __restrict__ chunk_start, int n,
                                                          uint32_t ntune, uint32_t total_chunks, uint32_t nb_range)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if (blockIdx.x < ntune) {
        const int f = find_field(sample_start, n, blockIdx.x);
        const BatchField& F = fields[f];
        tune_sample<A>(reinterpret_cast<float*>(smem), &F.tmap, F.g, F.x, F.cands, blockIdx.x - __ldg(sample_start + f),
                       0, 1, F.stride, F.m, F.err, &F.tickets[1], F.hdr, F.tma_bytes, (F.flags & kFlagTma) != 0);
        return;
    }
    batch_range_items(fields, chunk_start, n, total_chunks, blockIdx.x - ntune, nb_range);
}

// After the auto-tuner: each field's constants, status and level
// configuration from its header into its record.
__global__ void k_batch_gather(BatchField* __restrict__ fields)
{
    BatchField& F = fields[blockIdx.x];
    const hi_header* hdr = F.cur.out.hdr;
    const int tid = threadIdx.x;
    if (tid == 0) {
        F.cur.h.eb_f = hdr->eb_f;
        F.cur.h.ebx2_f = hdr->ebx2_f;
        F.cur.h.r_f = hdr->r_f;
        const uint32_t st = hdr->status;
        F.cur.skip = st != 0 && st != HI_ECAPACITY;
    }
    if (tid < HI_MAX_LEVELS) {
        const hi_level lv = hdr->level[tid];
        F.cur.lv[tid] = lv;
        F.cur.sel[tid] = perm_sel(lv);
    }
}

// Asynchronous copy of a field's record into a shared-memory slot (thread 0).
__device__ __forceinline__ void fetch_cur(BatchCur* dst, const BatchCur* src)
{
    static_assert(sizeof(BatchCur) % 16 == 0, "16-byte copies");
    for (int k = 0; k < (int)(sizeof(BatchCur) / 16); ++k) cp_async16(reinterpret_cast<char*>(dst) + 16 * k,
                                                                       reinterpret_cast<const char*>(src) + 16 * k);
}

// Thread 0 of a batched CTA, at iteration `it` on a tile of field f: takes
// the next work item from the queue (in queue order the CTAs in flight work
// on neighbouring tiles, which share faces and DRAM pages; that outweighs
// the cost of changing field), decodes it into slot (it + 1) & 1, starts the
// asynchronous copy of its field's record into `nslot` when that field is
// not f, and starts its box: into `other` with two buffers, into L2 with one.
template <int A>
__device__ __forceinline__ void batch_next(const BatchField* __restrict__ fields,
                                           const uint32_t* __restrict__ head_start,
                                           const uint32_t* __restrict__ shell_start, int n, uint32_t total_head,
                                           uint32_t total, uint32_t* queue, int it, bool dbuf, int f, float* other,
                                           uint64_t* s_mbar, int* s_next, int* s_tf, int* s_tma, uint32_t* s_tb,
                                           TileInfo* s_ti, BatchCur* nslot)
{
    const int buf = dbuf ? (it & 1) : 0;
    const uint32_t nx = gridDim.x + atomicAdd(queue, 1u);
    *s_next = (int)(nx < total ? nx : total);
    if (nx >= total) return;
    int pos;
    const int fn = batch_locate(fields, head_start, shell_start, n, total_head, nx, &pos);
    const BatchField& F = fields[fn];
    const TileInfo tn = tile_info<A>(F.g, pos);
    const int nb = (it + 1) & 1;
    const bool tma = (F.flags & kFlagTma) != 0;
    s_tf[nb] = fn;
    s_ti[nb] = tn;
    s_tma[nb] = tma;
    s_tb[nb] = F.tma_bytes;
    if (fn != f) fetch_cur(nslot, &F.cur);
    if (tma) {
        if (dbuf) {
            mbar_arrive_expect_tx(&s_mbar[buf ^ 1], F.tma_bytes);
            tma_load_3d(other, &F.tmap, tn.o[2], tn.o[1], tn.o[0], &s_mbar[buf ^ 1]);
        } else {
            tma_prefetch_3d(&F.tmap, tn.o[2], tn.o[1], tn.o[0]);
        }
    }
}

template <int A>
__global__ void __launch_bounds__(kMaxThreads, 5)
    k_compress_batch(const BatchField* __restrict__ fields, const uint32_t* __restrict__ head_start,
                     const uint32_t* __restrict__ shell_start, const int n, const uint32_t total_head,
                     const uint32_t total, uint32_t* __restrict__ queue, const int dbuf_flag)
{
    using Lw = Lay<A>;
    extern __shared__ __align__(128) unsigned char smem[];
    const bool dbuf = dbuf_flag != 0;
    const int vb_bytes = vbuf_bytes<A>(A + 1);
    float* const vbuf0 = reinterpret_cast<float*>(smem);
    float* const vbuf1 = reinterpret_cast<float*>(smem + (dbuf ? vb_bytes : 0));
    uint8_t* cs = smem + (dbuf ? 2 : 1) * vb_bytes;
    uint16_t* hc = A <= 16 ? nullptr : reinterpret_cast<uint16_t*>(cs + round128((A + 1) * Lw::P * Lw::CXC));
    __shared__ uint32_t s_hist[256];
    __shared__ __align__(8) uint64_t s_mbar[2];
    __shared__ BatchCur s_cur[2];  // the current field's record; the next field's, arriving
    __shared__ int s_next;
    __shared__ int s_tf[2];       // field of this work item and of the next
    __shared__ int s_tma[2];      // staged by TMA
    __shared__ uint32_t s_tb[2];  // bytes of its TMA box
    __shared__ TileInfo s_ti[2];

    const int tid = threadIdx.x;
    for (int i = tid; i < 256; i += blockDim.x) s_hist[i] = 0;
    for (int k = 0; hc && k < kHistBins; ++k) hc[k * blockDim.x + tid] = 0;
    if (tid == 0) {
        mbar_init(&s_mbar[0], 1);
        mbar_init(&s_mbar[1], 1);
        fence_mbar_init();
        if (blockIdx.x < total) {
            int pos;
            const int f = batch_locate(fields, head_start, shell_start, n, total_head, blockIdx.x, &pos);
            const BatchField& F = fields[f];
            const TileInfo t0 = tile_info<A>(F.g, pos);
            s_tf[0] = f;
            s_ti[0] = t0;
            s_tma[0] = (F.flags & kFlagTma) != 0;
            s_tb[0] = F.tma_bytes;
            if (s_tma[0]) {
                mbar_arrive_expect_tx(&s_mbar[0], F.tma_bytes);
                tma_load_3d(vbuf0, &F.tmap, t0.o[2], t0.o[1], t0.o[0], &s_mbar[0]);
            }
            fetch_cur(&s_cur[0], &F.cur);
            cp_async_wait_all();
        }
    }
    __syncthreads();

    int cur = s_tf[0];
    int sl = 0;       // slot of the current field's record
    uint32_t ph = 0;  // bit b: phase of buffer b's barrier
    int it = 0;
    for (uint32_t w = blockIdx.x; w < total; ++it) {
        const int buf = dbuf ? (it & 1) : 0;
        float* v = buf ? vbuf1 : vbuf0;
        const int f = s_tf[it & 1];
        const bool tma_here = s_tma[it & 1] != 0;
        const TileInfo ti = s_ti[it & 1];
        if (tid == 0 && !dbuf && it > 0 && tma_here) {  // one buffer: it is free again
            mbar_arrive_expect_tx(&s_mbar[0], s_tb[it & 1]);
            tma_load_3d(v, &fields[f].tmap, ti.o[2], ti.o[1], ti.o[0], &s_mbar[0]);
        }
        if (f != cur) {  // a new field: flush the last one's histogram; its record is in the other slot
            // (the last iteration's closing barrier ordered every count of it)
            if (s_cur[sl].hist) hist_flush_to(hc, s_hist, s_cur[sl].hist);
            if (tid == 0) cp_async_wait_all();
            __syncthreads();
            sl ^= 1;
            cur = f;
        }
        const BatchCur& C = s_cur[sl];
        if (tid == 0)
            batch_next<A>(fields, head_start, shell_start, n, total_head, total, queue, it, dbuf, f,
                          buf ? vbuf0 : vbuf1, s_mbar, &s_next, s_tf, s_tma, s_tb, s_ti, &s_cur[sl ^ 1]);
        if (tid < 8) {  // anchors keep the zero-error code
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            if (a0 * A <= ti.e[0] && a1 * A <= ti.e[1] && a2 * A <= ti.e[2])
                cs[a0 * A * Lw::CYC + a1 * A * Lw::CXC + a2 * A] = (uint8_t)kRadius;
        }
        if (tma_here) {
            const bool ok = mbar_wait(&s_mbar[buf], (ph >> buf) & 1u, kSpinLimit);
            ph ^= 1u << buf;
            if (!__syncthreads_and(ok)) {
                // copies this CTA issued may still be in flight: stay until they land
                if (tid == 0) set_status(&C.out.hdr->status, HI_ETIMEOUT);
                drain_wait(&s_mbar[buf], ((ph >> buf) & 1u) ^ 1u);
                if (dbuf && s_next < (int)total && s_tma[(it + 1) & 1])
                    drain_wait(&s_mbar[buf ^ 1], (ph >> (buf ^ 1)) & 1u);
                if (tid == 0) cp_async_wait_all();
                __syncthreads();
                return;
            }
        } else {
            load_tile_plain<A>(v, C.x, C.g, ti);
            __syncthreads();
            const int nf = s_tf[(it + 1) & 1];
            if (s_next < (int)total && !s_tma[(it + 1) & 1])
                prefetch_rows_l2<A>(fields[nf].x, 4, fields[nf].g, s_ti[(it + 1) & 1]);
        }
        const int next = s_next;
        if (!C.skip) {
            const bool full_ok = HasFull<A>::value && C.g.n[0] > 1 && C.g.n[1] > 1 && C.g.n[2] > 1;
            compress_tile<A>(C.g, ti, v, cs, hc, s_hist, C.sel, C.lv, C.h, full_ok, C.out);
        }
        if ((it % kHistFoldTiles) == kHistFoldTiles - 1) hist_fold(hc, s_hist);
        fence_proxy_async_smem();
        __syncthreads();
        w = (uint32_t)next;
    }
    if (blockIdx.x < total && s_cur[sl].hist) hist_flush(hc, s_hist, s_cur[sl].hist);
    if (tid == 0) cp_async_wait_all();
}

cudaError_t launch_batch_gather(const BatchLaunch& b, cudaStream_t st)
{
    k_batch_gather<<<b.n, 32, 0, st>>>(const_cast<BatchField*>(b.fields));
    return cudaGetLastError();
}

cudaError_t launch_batch_prologue(const BatchLaunch& b, cudaStream_t st)
{
    k_batch_prologue<<<b.n, 256, 0, st>>>(b.fields, b.queue);
    return cudaGetLastError();
}

template <int A>
static cudaError_t launch_batch_range_tune_t(const BatchLaunch& b, cudaStream_t st)
{
    using TG = TileGeom<A>;
    const size_t smem = b.total_samples ? (size_t)(A + 1) * TG::P * TG::PX * 4 : 0;
    auto kern = k_batch_range_tune<A>;
    cudaError_t e = set_max_smem(kern, smem);
    if (e != cudaSuccess) return e;
    uint32_t nb_range = (uint32_t)b.num_sms * 8;
    if (nb_range > b.total_chunks) nb_range = b.total_chunks;
    const uint32_t ntune = b.total_samples;
    kern<<<ntune + nb_range, 256, smem, st>>>(b.fields, b.sample_start, b.chunk_start, b.n, ntune, b.total_chunks,
                                             nb_range);
    return cudaGetLastError();
}

cudaError_t launch_batch_range_tune(const BatchLaunch& b, cudaStream_t st)
{
    if (b.total_samples == 0 && b.total_chunks == 0) return cudaSuccess;
    switch (b.A) {
    case 8: return launch_batch_range_tune_t<8>(b, st);
    case 16: return launch_batch_range_tune_t<16>(b, st);
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
    kern<<<grid, b.threads, smem, st>>>(b.fields, b.tile_start, b.shell_start, b.n, b.total_head, b.total_tiles,
                                        b.queue, dbuf ? 1 : 0);
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
