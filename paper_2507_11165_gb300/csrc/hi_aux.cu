// hi_aux.cu -- the smaller stages around the predict/quantize kernel:
//   * header set-up (and the absolute error bound's constants),
//   * the value range for the value-range-relative bound (Sec. 6.1.4) and the
//     float32 quantizer constants derived from it (Eq. 1),
//   * the outlier scatter that precedes reconstruction,
//   * the auto-tuner (Sec. 5.1.3): per-level error of every spline and
//     dimension sequence on uniformly sampled blocks, then the argmin.
#include <cstdint>

#include "hi_aux_dev.cuh"

namespace hi {

__global__ void k_prologue(hi_header* hdr, const hi_params p, uint64_t n_anchors, uint64_t out_cap,
                           uint32_t n_levels, uint32_t* hist, uint32_t* ticket, uint32_t* queue)
{
    prologue_fill(hdr, p, n_anchors, out_cap, n_levels, hist, ticket, ticket ? ticket + 2 : nullptr, queue);
}

// Value range over the finite values: one grid-strided streaming read; the
// last CTA to finish (ticket) folds the per-CTA partials and derives eps.
__global__ void __launch_bounds__(512) k_range(const float* __restrict__ x, int64_t N, float2* partials,
                                               uint32_t* ticket, hi_header* hdr)
{
    range_block(x, N, partials, blockIdx.x, gridDim.x, ticket, hdr);
}

// A field's auto-tune samples are each split over this many blocks (the
// candidates of a sample dealt out round robin): enough blocks to run beside
// the range pass, each tile loaded by few of them.
constexpr int kTuneGroups = 4;

// The value range and the auto-tuner in one launch: they do not depend on
// each other (the tuner's errors are open-loop, without eps), and the
// tuner's latency-bound blocks (first in the grid) run beside the range
// pass's streaming read.  Blocks [0, m * kTuneGroups): auto-tune, a sample
// and a group of candidates each; the next nb_range blocks: the range pass.
template <int A>
__global__ void __launch_bounds__(256) k_range_tune(const __grid_constant__ CUtensorMap tmap, const FieldGeo g,
                                                    const float* __restrict__ x, const TuneCands cands, int stride,
                                                    int m, double* __restrict__ err, uint32_t* tune_ticket,
                                                    const uint32_t tma_bytes, const int use_tma, float2* partials,
                                                    int nb_range, uint32_t* range_ticket, hi_header* hdr)
{
    extern __shared__ __align__(128) unsigned char smem[];
    if ((int)blockIdx.x < m * kTuneGroups) {
        tune_sample<A>(reinterpret_cast<float*>(smem), &tmap, g, x, cands, blockIdx.x / kTuneGroups,
                       blockIdx.x % kTuneGroups, kTuneGroups, stride, m, err, tune_ticket, hdr, tma_bytes,
                       use_tma != 0);
        return;
    }
    range_block(x, g.N, partials, (int)blockIdx.x - m * kTuneGroups, nb_range, range_ticket, hdr);
}

// Outlier values go to their place in the output before reconstruction reads
// them there (code 0 means "take the stored value").
__global__ void k_scatter(const uint32_t* __restrict__ idx, const float* __restrict__ val, uint64_t cap,
                          const hi_header* __restrict__ hdr, int64_t N, float* __restrict__ out,
                          uint32_t* __restrict__ status, uint32_t* __restrict__ queue)
{
    const uint64_t n_all = hdr->n_outliers;
    const uint64_t n = n_all < cap ? n_all : cap;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        *queue = 0;  // the reconstruction kernel's tile queue
        if (hdr->magic != HI_MAGIC) set_status(status, HI_ECORRUPT);
        if (n_all > cap) set_status(status, HI_ECAPACITY);
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t k = idx[i];
        if ((int64_t)k < N)
            out[k] = val[i];
        else
            set_status(status, HI_ECORRUPT);
    }
}

template <int A>
__global__ void __launch_bounds__(256) k_tune(const __grid_constant__ CUtensorMap tmap, const FieldGeo g,
                                              const float* __restrict__ x, const TuneCands cands, int stride,
                                              double* __restrict__ err, uint32_t* ticket,
                                              hi_header* __restrict__ hdr, const uint32_t tma_bytes, const int use_tma)
{
    extern __shared__ __align__(128) unsigned char smem[];
    tune_sample<A>(reinterpret_cast<float*>(smem), &tmap, g, x, cands, blockIdx.x / kTuneGroups,
                   blockIdx.x % kTuneGroups, kTuneGroups, stride, gridDim.x / kTuneGroups, err, ticket, hdr, tma_bytes,
                   use_tma != 0);
}

cudaError_t launch_prologue(hi_header* hdr, const hi_params& p, uint64_t n_anchors, uint64_t out_cap,
                            uint32_t n_levels, uint32_t* hist, uint32_t* ticket, uint32_t* queue, cudaStream_t st)
{
    k_prologue<<<1, 256, 0, st>>>(hdr, p, n_anchors, out_cap, n_levels, hist, ticket, queue);
    return cudaGetLastError();
}

cudaError_t launch_range(const float* x, int64_t N, float2* partials, int nblocks, uint32_t* ticket,
                         hi_header* hdr, cudaStream_t st)
{
    k_range<<<nblocks, 512, 0, st>>>(x, N, partials, ticket, hdr);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const uint32_t* idx, const float* val, uint64_t cap, const hi_header* hdr, int64_t N,
                           float* out, uint32_t* status, uint32_t* queue, cudaStream_t st)
{
    k_scatter<<<256, 256, 0, st>>>(idx, val, cap, hdr, N, out, status, queue);
    return cudaGetLastError();
}

template <int A>
static cudaError_t launch_tune_t(const TuneLaunch& t, cudaStream_t st)
{
    using TG = TileGeom<A>;
    const size_t smem = (size_t)t.g.b0 * TG::P * TG::PX * 4;
    auto kern = k_tune<A>;
    cudaError_t e = set_max_smem(kern, smem);
    if (e != cudaSuccess) return e;
    kern<<<t.m * kTuneGroups, 256, smem, st>>>(t.tmap, t.g, t.x, t.cands, t.stride, t.err, t.ticket, t.hdr,
                                               t.tma_bytes, t.use_tma ? 1 : 0);
    return cudaGetLastError();
}

template <int A>
static cudaError_t launch_range_tune_t(const TuneLaunch& t, float2* partials, int nb_range, uint32_t* range_ticket,
                                       cudaStream_t st)
{
    using TG = TileGeom<A>;
    const size_t smem = (size_t)t.g.b0 * TG::P * TG::PX * 4;
    auto kern = k_range_tune<A>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    kern<<<t.m * kTuneGroups + nb_range, 256, smem, st>>>(t.tmap, t.g, t.x, t.cands, t.stride, t.m, t.err,
                                                             t.ticket, t.tma_bytes, t.use_tma ? 1 : 0, partials,
                                                             nb_range, range_ticket, t.hdr);
    return cudaGetLastError();
}

cudaError_t launch_range_tune(int A, const TuneLaunch& t, float2* partials, int nb_range, uint32_t* range_ticket,
                              cudaStream_t st)
{
    switch (A) {
    case 2: return launch_range_tune_t<2>(t, partials, nb_range, range_ticket, st);
    case 4: return launch_range_tune_t<4>(t, partials, nb_range, range_ticket, st);
    case 8: return launch_range_tune_t<8>(t, partials, nb_range, range_ticket, st);
    case 16: return launch_range_tune_t<16>(t, partials, nb_range, range_ticket, st);
    case 32: return launch_range_tune_t<32>(t, partials, nb_range, range_ticket, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_tune(int A, const TuneLaunch& t, cudaStream_t st)
{
    switch (A) {
    case 2: return launch_tune_t<2>(t, st);
    case 4: return launch_tune_t<4>(t, st);
    case 8: return launch_tune_t<8>(t, st);
    case 16: return launch_tune_t<16>(t, st);
    case 32: return launch_tune_t<32>(t, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace hi
