// hi_internal.h -- launch descriptors shared between the C ABI (hi_api.cu)
// and the kernel translation units.  Not part of the public interface.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cuda.h>
#include <cuda_runtime.h>

#include "../../include/hi.h"
#include "hi_device.cuh"

namespace hi {

enum : int {
    kFlagTma = 1,       // stage tiles with TMA (strides meet the 16-byte rules)
    kFlagVecCodes = 2,  // code rows may be stored as 8/16-byte vectors
    kFlagVecOut = 4,    // float rows may be stored as 16-byte vectors
    kFlagDoubleBuf = 8, // two tile buffers fit in shared memory: prefetch the next tile
};

struct CompressLaunch {
    CUtensorMap tmap;
    FieldGeo g;
    const float* x;
    uint8_t* codes;
    float* anchors;
    uint32_t* out_idx;
    float* out_val;
    uint64_t out_cap;
    uint32_t* hist;
    float* recon;
    hi_header* hdr;
    uint32_t* queue;  // tile queue counter, zero at launch
    uint32_t tma_bytes;
    int flags;
    int threads;
    int buffers;   // 0 = two when they fit, 1 = one, 2 = two
    int num_sms;
    int max_ctas;  // 0 = occupancy-limited persistent grid
};

struct DecompressLaunch {
    CUtensorMap cmap;
    FieldGeo g;
    const uint8_t* codes;
    const float* anchors;
    float* out;
    const hi_header* hdr;
    uint32_t* status;
    uint32_t* queue;  // tile queue counter, zero at launch
    uint32_t tma_bytes;
    int flags;
    int threads;
    int buffers;
    int num_sms;
    int max_ctas;
};

// Auto-tune candidates of one level.
struct TuneCands {
    int ncfg;
    int nperm;
    uint8_t interp[12];
    uint8_t order[12][3];
};

cudaError_t launch_compress(int A, const CompressLaunch& c, cudaStream_t st);
cudaError_t launch_decompress(int A, const DecompressLaunch& c, cudaStream_t st);
size_t compress_smem_bytes(int A, int b0);

// hi_aux.cu
cudaError_t launch_prologue(hi_header* hdr, const hi_params& p, uint64_t n_anchors, uint64_t out_cap,
                            uint32_t n_levels, uint32_t* hist, uint32_t* ticket, uint32_t* queue, cudaStream_t st);
cudaError_t launch_range(const float* x, int64_t N, float2* partials, int nblocks, uint32_t* ticket,
                         hi_header* hdr, cudaStream_t st);
cudaError_t launch_scatter(const uint32_t* idx, const float* val, uint64_t cap, const hi_header* hdr, int64_t N,
                           float* out, uint32_t* status, uint32_t* queue, cudaStream_t st);
struct TuneLaunch {
    CUtensorMap tmap;
    FieldGeo g;
    const float* x;
    TuneCands cands;
    int m, stride;
    double* err;
    uint32_t* ticket;
    hi_header* hdr;
    uint32_t tma_bytes;
    bool use_tma;
};
cudaError_t launch_tune(int A, const TuneLaunch& t, cudaStream_t st);

constexpr int kRangeBlocks = 1024;

}  // namespace hi
