// hi_compress_pipe.cu -- the fused interpolation-predict + quantize step as a
// two-stage pipeline per CTA (cuSZ-Hi, arXiv 2507.11165, Sec. 3.2,
// Sec. 5.1.1-5.1.2, Sec. 5.2.1), for 3D fields whose tiles TMA can stage.
//
// The coarse levels of a tile (strides A/2 .. 2: the points on its even
// sub-lattice, about a seventh of them) are many small passes, each a
// handful of lines; run by the whole CTA they leave it mostly idle between
// barriers.  Here a CTA has five warps:
//   * warp 0 takes tiles from the queue, stages tile j+1 with TMA into one of
//     two tile buffers and runs its coarse levels (warp barriers only);
//   * warps 1..4 run the finest level (stride 1, six sevenths of the points)
//     of tile j in the other buffer and its epilogue (codes, histogram,
//     anchor, outliers), synchronised by a named barrier.
// The two stages hand buffers over through mbarriers: ready[b] (the coarse
// levels of the tile in buffer b are done, 32 arrivals), freeF[b] (tile
// buffer b may be overwritten: right after the finest level, so that the next
// copy overlaps the epilogue) and freeC[b] (code box b may be overwritten,
// after the epilogue), 128 arrivals each.  Every wait is bounded; a stage that
// gives up records HI_ETIMEOUT and stops the pipeline, and a warp that issued
// a copy waits for it to land before the CTA moves on.
//
// The fast tiles (below the last block along every dim) are the head of the
// tile order; the pipeline takes them by static stride over the CTAs.  Then
// every warp of the CTA takes the remaining tiles (the field's last blocks)
// from the queue one at a time with the per-tile path of
// hi_compress_tile.cuh.
#include "hi_compress_tile.cuh"
#include "hi_fast.cuh"

namespace hi {

constexpr int kPipeThreads = 160;
// Warp 0 pulls the box of the tile this many steps ahead into L2 (a bulk
// tensor prefetch, no shared memory): with two tile buffers per CTA the
// loads alone would keep too few bytes in flight to cover DRAM latency.
constexpr int kPipePrefetch = 3;
using CoarseGrp = Grp<32, 0, -1>;
using FineGrp = Grp<128, 32, 1>;

struct PipeJob {
    TileInfo ti;
    int pos;  // queue position of the tile in this buffer; -1: the pipeline is over
    int bad;  // a coarse-level point of the tile is an outlier
};

// Shared-memory layout: two tile buffers, two owned code boxes (A^3 bytes);
// the per-tile path after the pipeline keeps its 16-bit histogram counters in
// the second tile buffer, or behind the code boxes when they do not fit there.
constexpr int kPipeHcBytes = kHistBins * kPipeThreads * (int)sizeof(uint16_t);

template <int A>
__host__ __device__ constexpr int pipe_hc_extra(int b0)
{
    return vbuf_bytes<A>(b0) >= kPipeHcBytes ? 0 : kPipeHcBytes;
}

template <int A>
size_t pipe_smem_bytes(int b0)
{
    return 2 * (size_t)vbuf_bytes<A>(b0) + 2 * (size_t)round128(A * A * A) + (size_t)pipe_hc_extra<A>(b0);
}

// Arrive on an mbarrier (release at CTA scope by default).
__device__ __forceinline__ void mbar_arrive(uint64_t* mbar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(mbar)) : "memory");
}

template <int A>
__global__ void __launch_bounds__(kPipeThreads, 4)
    k_compress_pipe(const __grid_constant__ CUtensorMap tmap, const FieldGeo g, const float* __restrict__ x,
                    uint8_t* __restrict__ codes, float* __restrict__ anchors, uint32_t* __restrict__ out_idx,
                    float* __restrict__ out_val, const uint64_t out_cap, uint32_t* __restrict__ hist_g,
                    float* __restrict__ recon_g, hi_header* __restrict__ hdr, uint32_t* __restrict__ queue,
                    const uint32_t tma_bytes, const int flags)
{
    using Lw = Lay<A>;
    constexpr int L = TileGeom<A>::L;
    extern __shared__ __align__(128) unsigned char smem[];
    const int vb_bytes = vbuf_bytes<A>(g.b0);
    float* const F0 = reinterpret_cast<float*>(smem);
    float* const F1 = reinterpret_cast<float*>(smem + vb_bytes);
    uint8_t* const C0 = smem + 2 * vb_bytes;
    uint8_t* const C1 = C0 + round128(A * A * A);
    __shared__ uint32_t s_hist[256];
    __shared__ __align__(8) uint64_t s_tma[2];
    __shared__ __align__(8) uint64_t s_ready[2];
    __shared__ __align__(8) uint64_t s_freeF[2];
    __shared__ __align__(8) uint64_t s_freeC[2];
    __shared__ __align__(8) uint64_t s_mrest;
    __shared__ hi_level s_lv[HI_MAX_LEVELS];
    __shared__ int s_sel[HI_MAX_LEVELS];
    __shared__ PipeJob s_job[2];
    __shared__ int s_nx[2];  // queue positions of the per-tile path, alternating

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    {   // an earlier stage failed (bad range, device-side EINVAL): leave outputs untouched
        const uint32_t st = hdr->status;
        if (__syncthreads_or(st != 0 && st != HI_ECAPACITY)) return;
    }
    Hot h;
    h.eb_f = hdr->eb_f;
    h.ebx2_f = hdr->ebx2_f;
    h.r_f = hdr->r_f;
    const FastC fc = fast_consts(h);
    const bool hist_on = hist_g != nullptr;
    for (int i = tid; i < 256; i += blockDim.x) s_hist[i] = 0;
    if (tid < HI_MAX_LEVELS) {
        s_lv[tid] = hdr->level[tid];
        s_sel[tid] = perm_sel(s_lv[tid]);
    }
    if (tid == 0) {
        for (int b = 0; b < 2; ++b) {
            mbar_init(&s_tma[b], 1);
            mbar_init(&s_ready[b], 32);
            mbar_init(&s_freeF[b], 128);
            mbar_init(&s_freeC[b], 128);
        }
        mbar_init(&s_mrest, 1);
        fence_mbar_init();
        prefetch_tmap(&tmap);
    }
    __syncthreads();
    const bool full_ok = HasFull<A>::value && g.n[0] > 1 && g.n[1] > 1 && g.n[2] > 1;
    const int n_fast = full_ok ? g.ni[0] * g.ni[1] * g.ni[2] : 0;
    uint32_t hacc = 0;  // fine threads: histogram bins 126..129, a byte each

    if (warp == 0) {
        // ---- producer and coarse levels: the fast tiles (the head of the
        // queue order) by static stride, all of equal cost
        for (int j = 0;; ++j) {
            const int b = j & 1;
            const uint32_t k = (uint32_t)j >> 1;
            float* v = b ? F1 : F0;
            uint8_t* cs = b ? C1 : C0;
            const int pos = (int)blockIdx.x + j * (int)gridDim.x;
            bool stop = false;
            // the fine stage is done with the tile buffer of the tile two back --
            // waited for even when no tile follows, so that ready[b] is never
            // posted before the fine stage has taken its previous phase
            if (j >= 2) {
                const bool ok = mbar_wait(&s_freeF[b], (k - 1) & 1u, kSpinLimit);
                if (!__all_sync(0xffffffffu, ok)) {
                    if (lane == 0) set_status(&hdr->status, HI_ETIMEOUT);
                    stop = true;
                }
            }
            stop = stop || pos >= n_fast;
            TileInfo ti{};
            if (!stop) ti = tile_info<A>(g, pos);
            if (stop || !fast_tile<A>(full_ok, ti)) {
                if (lane == 0) s_job[b].pos = -1;
                __syncwarp();
                mbar_arrive(&s_ready[b]);
                break;
            }
            if (lane == 0) {
                mbar_arrive_expect_tx(&s_tma[b], tma_bytes);
                tma_load_3d(v, &tmap, ti.o[2], ti.o[1], ti.o[0], &s_tma[b]);
                if (j == 0)  // the first steps' boxes
                    for (int q = 1; q < kPipePrefetch; ++q) {
                        const int pq = pos + q * (int)gridDim.x;
                        if (pq < n_fast) tma_l2_prefetch(&tmap, g, pq, A);
                    }
                const int pf = pos + kPipePrefetch * (int)gridDim.x;
                if (pf < n_fast) tma_l2_prefetch(&tmap, g, pf, A);
            }
            // ... and with the code box of the tile two back (its epilogue)
            const bool okc = j < 2 || mbar_wait(&s_freeC[b], (k - 1) & 1u, kSpinLimit);
            const bool ok = okc && mbar_wait(&s_tma[b], k & 1u, kSpinLimit);
            if (lane == 0 && ok) cs[0] = (uint8_t)kRadius;  // the owned anchor keeps the zero-error code
            if (!__all_sync(0xffffffffu, ok)) {
                // the copy may still be in flight: stay until it lands
                if (lane == 0) set_status(&hdr->status, HI_ETIMEOUT);
                drain_wait(&s_tma[b], k & 1u);
                if (lane == 0) s_job[b].pos = -1;
                __syncwarp();
                mbar_arrive(&s_ready[b]);
                break;
            }
            bool bad = slevels<A, L - 1, 1, true, CoarseGrp>(s_sel, v, cs, h);
            bad = __any_sync(0xffffffffu, bad);
            if (lane == 0) {
                s_job[b].ti = ti;
                s_job[b].pos = pos;
                s_job[b].bad = bad ? 1 : 0;
            }
            __syncwarp();
            mbar_arrive(&s_ready[b]);
        }
    } else {
        // ---- finest level and epilogue
        const int ft = FineGrp::tid();
        int nfast = 0;
        for (int j = 0;; ++j) {
            const int b = j & 1;
            const uint32_t k = (uint32_t)j >> 1;
            float* v = b ? F1 : F0;
            uint8_t* cs = b ? C1 : C0;
            const bool ok = mbar_wait(&s_ready[b], k & 1u, kSpinLimit);
            if (FineGrp::sync_or(!ok)) {
                if (ft == 0) set_status(&hdr->status, HI_ETIMEOUT);
                break;
            }
            const int pos = s_job[b].pos;
            if (pos < 0) break;
            const TileInfo ti = s_job[b].ti;
            const bool cbad = s_job[b].bad != 0;
            const bool bad = flevel_dispatch<A, 1, true, FineGrp>(s_sel[0], v, cs, fc, h);
            const bool any_out = FineGrp::sync_or(bad) || cbad;
            if (ft == 0) {
                const int64_t ai = ((int64_t)(ti.o[0] / A) * g.na[1] + ti.o[1] / A) * g.na[2] + ti.o[2] / A;
                anchors[ai] = v[0];
                if (hist_on) atomicSub(&s_hist[kRadius], 1u);  // the anchor is not predicted
            }
            // the tile buffer goes back to the producer (unless the reconstruction
            // is an output): order this stage's writes to it before the TMA that
            // overwrites it
            if (!recon_g) {
                fence_proxy_async_smem();
                mbar_arrive(&s_freeF[b]);
            }
            fast_codes_out<A, FineGrp>(g, ti, cs, codes, (flags & kFlagVecCodes) != 0, hist_on, hacc, s_hist);
            if (any_out) fast_outliers<A, FineGrp>(g, ti, cs, x, hdr, out_idx, out_val, out_cap);
            if (recon_g) {
                for (int i = ft; i < A * A * A; i += FineGrp::T) {
                    const int c0 = i / (A * A), c1 = (i / A) % A, c2 = i % A;
                    recon_g[((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2] + c2] =
                        v[c0 * Lw::PY + c1 * Lw::PX + c2];
                }
            }
            if (hist_on && ++nfast % kFastFlush == 0) fast_hist_flush(hacc, s_hist);
            if (recon_g) {
                fence_proxy_async_smem();
                mbar_arrive(&s_freeF[b]);
            }
            mbar_arrive(&s_freeC[b]);
        }
    }
    fence_proxy_async_smem();
    __syncthreads();
    if (hist_on) fast_hist_flush(hacc, s_hist);

    // ---- the remaining tiles (edge tiles), one at a time by the whole CTA
    uint16_t* hc = reinterpret_cast<uint16_t*>(pipe_hc_extra<A>(g.b0) ? C0 + 2 * round128(A * A * A)
                                                                      : reinterpret_cast<uint8_t*>(F1));
    if (hist_on)
        for (int q = 0; q < kHistBins; ++q) hc[q * blockDim.x + tid] = 0;
    if (tid == 0) s_nx[0] = n_fast + (int)atomicAdd(queue, 1u);
    const bool failed = __syncthreads_or(hdr->status == HI_ETIMEOUT);
    int tile = failed ? g.ntiles : s_nx[0];
    uint32_t ph = 0;
    int nslow = 0, it = 0;
    while (tile < g.ntiles) {
        const TileInfo ti = tile_info<A>(g, tile);
        float* v = F0;
        uint8_t* cs = C0;
        if (tid == 0) {
            tma_issue(v, &tmap, g, tile, A, &s_mrest, tma_bytes);
            const int nx = n_fast + (int)atomicAdd(queue, 1u);
            s_nx[(it + 1) & 1] = nx;
            if (nx < g.ntiles) tma_l2_prefetch(&tmap, g, nx, A);  // waits in L2 until this tile is done
        }
        if (tid < 8) {  // anchors keep the zero-error code
            const int a0 = (tid >> 2) & 1, a1 = (tid >> 1) & 1, a2 = tid & 1;
            if (a0 * A <= ti.e[0] && a1 * A <= ti.e[1] && a2 * A <= ti.e[2])
                cs[a0 * A * Lw::CYC + a1 * A * Lw::CXC + a2 * A] = (uint8_t)kRadius;
        }
        const bool ok = mbar_wait(&s_mrest, ph, kSpinLimit);
        if (!__syncthreads_and(ok)) {
            if (tid == 0) set_status(&hdr->status, HI_ETIMEOUT);
            drain_wait(&s_mrest, ph);
            __syncthreads();
            break;
        }
        ph ^= 1u;
        const int next = s_nx[(it + 1) & 1];
        const CompressOut out{codes, anchors, out_idx, out_val, out_cap, recon_g, hdr,
                              (flags & kFlagVecCodes) != 0, hist_on};
        compress_tile<A>(g, ti, v, cs, hc, s_hist, s_sel, s_lv, h, full_ok, out);
        if (hist_on && ++nslow % kHistFoldTiles == 0) hist_fold(hc, s_hist);
        fence_proxy_async_smem();
        __syncthreads();
        tile = next;
        ++it;
    }
    if (hist_on) hist_flush(hc, s_hist, hist_g);
}

template <int A>
static cudaError_t launch_pipe_t(const CompressLaunch& c, cudaStream_t st)
{
    auto kern = k_compress_pipe<A>;
    // the per-tile path after the pipeline keeps its codes in the two code
    // boxes and its histogram counters in the second tile buffer
    static_assert(2 * round128(A * A * A) >= (A + 1) * (A + 1) * Lay<A>::CXC, "code staging of the per-tile path");
    const size_t smem = pipe_smem_bytes<A>(c.g.b0);
    int grid = 0;
    cudaError_t err = persistent_grid(kern, kPipeThreads, smem, c.num_sms, c.g.ntiles, c.max_ctas, &grid);
    if (err != cudaSuccess) return err;
    kern<<<grid, kPipeThreads, smem, st>>>(c.tmap, c.g, c.x, c.codes, c.anchors, c.out_idx, c.out_val, c.out_cap,
                                          c.hist, c.recon, c.hdr, c.queue, c.tma_bytes, c.flags);
    return cudaGetLastError();
}

cudaError_t launch_compress_pipe(int A, const CompressLaunch& c, cudaStream_t st)
{
    switch (A) {
    case 8: return launch_pipe_t<8>(c, st);
    case 16: return launch_pipe_t<16>(c, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hi
