// hi_compress.cu -- the fused interpolation-predict + quantize kernel of one
// field (cuSZ-Hi, arXiv 2507.11165, Sec. 3.2, Sec. 5.1.1-5.1.2, Sec. 5.2.1):
// persistent CTAs take tiles from a queue, stage them with TMA and run
// compress_tile (hi_compress_tile.cuh) on each.  With SEQ the codes also go
// to the reordered sequence of Sec. 5.2.2 (Eq. 3) from the same registers.
#include "hi_compress_tile.cuh"

namespace hi {

// ---------------------------------------------------------------------------
// Predict + quantize
// ---------------------------------------------------------------------------
template <int A, bool SEQ>
__global__ void __launch_bounds__(kMaxThreads, 7)
    k_compress(const __grid_constant__ CUtensorMap tmap, const FieldGeo g, const float* __restrict__ x,
               uint8_t* __restrict__ codes, float* __restrict__ anchors, uint32_t* __restrict__ out_idx,
               float* __restrict__ out_val, const uint64_t out_cap, uint32_t* __restrict__ hist_g,
               float* __restrict__ recon_g, hi_header* __restrict__ hdr, uint32_t* __restrict__ queue,
               const uint32_t tma_bytes, const int flags, uint8_t* __restrict__ seq,
               const __grid_constant__ SeqGeo sg)
{
    using Lw = Lay<A>;
    extern __shared__ __align__(128) unsigned char smem[];
    const bool dbuf = flags & kFlagDoubleBuf;
    const int vb_bytes = vbuf_bytes<A>(g.b0);
    float* const vbuf0 = reinterpret_cast<float*>(smem);
    float* const vbuf1 = reinterpret_cast<float*>(smem + (dbuf ? vb_bytes : 0));
    uint8_t* cs = smem + (dbuf ? 2 : 1) * vb_bytes;
    uint16_t* hc = A <= 16 ? nullptr : reinterpret_cast<uint16_t*>(cs + round128(g.b0 * Lw::P * Lw::CXC));  // [kHistBins][threads]
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
        for (int k = 0; hc && k < kHistBins; ++k) hc[k * blockDim.x + tid] = 0;
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
            if ((int)blockIdx.x < g.ntiles) tma_issue(vbuf0, &tmap, g, blockIdx.x, A, &s_mbar[0], tma_bytes);
        }
    }
    __syncthreads();
    const bool full_ok = HasFull<A>::value && g.n[0] > 1 && g.n[1] > 1 && g.n[2] > 1;

    int nslow = 0;

    // tiles after each CTA's first come from a queue in ascending order: the
    // load stays balanced (edge tiles cost more) and neighbouring tiles, which
    // share faces, are in flight together
    int it = 0;
    for (int tile = blockIdx.x; tile < g.ntiles; ++it) {
        const int buf = dbuf ? (it & 1) : 0;
        float* v = buf ? vbuf1 : vbuf0;
        const TileInfo ti = s_ti[it & 1];
        if (tid == 0) {
            // one buffer: this tile's copy first (the buffer is free again),
            // before the queue's round trip
            if (use_tma && !dbuf && it > 0) tma_issue(v, &tmap, g, tile, A, &s_mbar[0], tma_bytes);
            const int nx = (int)gridDim.x + (int)atomicAdd(queue, 1u);
            s_next = nx;
            if (nx < g.ntiles) s_ti[(it + 1) & 1] = tile_info<A>(g, nx);
            if (use_tma && dbuf && nx < g.ntiles)
                tma_issue(buf ? vbuf0 : vbuf1, &tmap, g, nx, A, &s_mbar[buf ^ 1], tma_bytes);
        }
        if (tid < 8) {  // anchors keep the zero-error code
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            if (a0 * A <= ti.e[0] && a1 * A <= ti.e[1] && a2 * A <= ti.e[2])
                cs[a0 * A * Lw::CYC + a1 * A * Lw::CXC + a2 * A] = (uint8_t)kRadius;
        }
        if (use_tma) {
            const bool ok = mbar_wait(&s_mbar[buf], dbuf ? ((it >> 1) & 1) : (it & 1), kSpinLimit);
            if (!__syncthreads_and(ok)) {
                // the copies this CTA issued may still be in flight: record the
                // status and stay until they have landed (or a longer bound ends)
                if (tid == 0) set_status(&hdr->status, HI_ETIMEOUT);
                drain_wait(&s_mbar[buf], dbuf ? ((it >> 1) & 1) : (it & 1));
                if (dbuf && s_next < g.ntiles) drain_wait(&s_mbar[buf ^ 1], ((it + 1) >> 1) & 1);
                __syncthreads();
                return;
            }
        } else {
            load_tile_plain<A>(v, x, g, ti);
            __syncthreads();
            if (s_next < g.ntiles) prefetch_rows_l2<A>(x, 4, g, s_ti[(it + 1) & 1]);
        }
        const int next = s_next;
        {
            const CompressOut out{codes, anchors, out_idx, out_val, out_cap, recon_g, hdr,
                                  (flags & kFlagVecCodes) != 0, hist_on};
            compress_tile<A, SEQ>(g, ti, v, cs, hc, s_hist, s_sel, s_lv, h, full_ok, out, seq, &sg);
            if (hist_on && ++nslow % kHistFoldTiles == 0) hist_fold(hc, s_hist);
        }
        // keep the buffers until every thread is done; order the generic-proxy
        // writes above before the TMA overwrite of this buffer
        fence_proxy_async_smem();
        __syncthreads();
        tile = next;
    }
    if (hist_on) hist_flush(hc, s_hist, hist_g);
}

template <int A, bool SEQ>
static cudaError_t launch_compress_t(const CompressLaunch& c, cudaStream_t st)
{
    auto kern = k_compress<A, SEQ>;
    const bool dbuf = c.buffers == 2 && fits_double(kern, compress_smem_t<A>(c.g.b0, true, c.threads));
    const size_t smem = compress_smem_t<A>(c.g.b0, dbuf, c.threads);
    int grid = 0;
    cudaError_t err = persistent_grid(kern, c.threads, smem, c.num_sms, c.g.ntiles, c.max_ctas, &grid);
    if (err != cudaSuccess) return err;
    kern<<<grid, c.threads, smem, st>>>(c.tmap, c.g, c.x, c.codes, c.anchors, c.out_idx, c.out_val, c.out_cap,
                                        c.hist, c.recon, c.hdr, c.queue, c.tma_bytes,
                                        c.flags | (dbuf ? kFlagDoubleBuf : 0), c.seq, c.sg);
    return cudaGetLastError();
}

cudaError_t launch_compress(int A, const CompressLaunch& c, cudaStream_t st)
{
    if (c.seq) {
        switch (A) {
        case 8: return launch_compress_t<8, true>(c, st);
        case 16: return launch_compress_t<16, true>(c, st);
        default: return cudaErrorInvalidValue;
        }
    }
    switch (A) {
    case 2: return launch_compress_t<2, false>(c, st);
    case 4: return launch_compress_t<4, false>(c, st);
    case 8: return launch_compress_t<8, false>(c, st);
    case 16: return launch_compress_t<16, false>(c, st);
    case 32: return launch_compress_t<32, false>(c, st);
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
