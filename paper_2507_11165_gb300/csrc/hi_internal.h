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

// Quantizer constants every point needs (Eq. 1), passed by value.
struct Hot {
    float eb_f, ebx2_f, r_f;
};

// Where one field's results go.  The single-field kernel passes its kernel
// parameters by value; the batched kernel passes a view of the current
// field's record in shared memory, read only after the level passes so that
// no pointer stays in a register across them.
struct CompressOut {
    uint8_t* codes;
    float* anchors;
    uint32_t* out_idx;
    float* out_val;
    uint64_t out_cap;
    float* recon;
    hi_header* hdr;
    bool vec_ok;   // code rows may be stored as vectors
    bool hist_on;  // count the histogram
};

// Constants of the reordered sequence (Sec. 5.2.2, Eq. 3) per level l of
// the stride-2^l subgrid: D1, D2 = its extents along dims 1 and 2, H12 and
// H2 = the all-even points of a plane and of a row, prefix = the points of
// the coarser levels.
struct SeqGeo {
    uint32_t D1[HI_MAX_LEVELS], D2[HI_MAX_LEVELS];
    uint32_t H12[HI_MAX_LEVELS], H2[HI_MAX_LEVELS];
    uint32_t prefix[HI_MAX_LEVELS];
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
    int buffers;   // 2: two tile buffers when they fit; otherwise one
    int num_sms;
    int max_ctas;  // 0 = occupancy-limited persistent grid
    uint8_t* seq;  // non-null: the codes also go to their places in the reordered sequence (A = 8 or 16,
                   // every row whole and stored as vectors, every run aligned to its length)
    SeqGeo sg;
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

// Auto-tune candidates of one level: the 1D sequences, then the
// multi-dimensional scheme (two or more active dims).
constexpr int kMaxCands = 14;

struct TuneCands {
    int ncfg;
    int nperm;
    uint8_t interp[kMaxCands];
    uint8_t order[kMaxCands][3];
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
cudaError_t launch_range_tune(int A, const TuneLaunch& t, float2* partials, int nb_range, uint32_t* range_ticket,
                              cudaStream_t st);

constexpr int kRangeBlocks = 1024;

// ---------------------------------------------------------------------------
// Batches: many fields in one launch per stage.  The host writes one
// BatchField per field into the workspace; every batched kernel finds the
// field of a work item by binary search over a prefix array.
// ---------------------------------------------------------------------------
constexpr int64_t kBatchChunk = 1 << 18;  // points per range work item

// What the predict-quantize kernel needs of a field: copied whole into
// shared memory (16-byte asynchronous copies) when a CTA moves to the field.
// The host fills the static part; after the auto-tuner, a gather launch
// copies the constants, the status and the level configuration from the
// field's header.
struct alignas(16) BatchCur {
    CompressOut out;
    FieldGeo g;
    const float* x;
    uint32_t* hist;
    Hot h;
    int flags;
    int skip;     // an earlier stage of this field failed: leave its outputs
    int full_ok;  // every dim active: whole tiles take the compile-time passes
    hi_level lv[HI_MAX_LEVELS];
    int sel[HI_MAX_LEVELS];
};

struct alignas(128) BatchField {
    CUtensorMap tmap;  // the field as (PX, A+1, b0) float boxes (when flags & kFlagTma)
    CUtensorMap cmap;  // its codes as (CX, A+1, b0) byte boxes (when dflags & kFlagTma)
    BatchCur cur;
    FieldGeo g;
    hi_params p;
    const float* x;
    uint8_t* codes;
    float* anchors;
    uint32_t* out_idx;
    float* out_val;
    uint64_t out_cap;
    uint32_t* hist;
    float* recon;
    hi_header* hdr;
    uint64_t n_anchors;
    float2* partials;   // range partials, one per chunk
    double* err;        // auto-tune sums [m][L][ncfg]
    uint32_t* tickets;  // [0] range, [1] auto-tune
    TuneCands cands;
    uint32_t n_levels;
    uint32_t tma_bytes;
    int flags;
    int m, stride;       // auto-tune samples (m = 0: levels given)
    uint32_t nchunks;    // range work items (0: absolute bound)
    uint32_t nint;       // tiles at the head of the field's queue order (whole 3D tiles first)
    float* out;          // reconstruction target of the batched decompression
    uint32_t ctma_bytes; // bytes of a code box
    int dflags;          // decompression: kFlagTma (code boxes), kFlagVecOut
};

struct BatchLaunch {
    const BatchField* fields;
    const uint32_t* tile_start;    // [n + 1] first work item of each field's head tiles (nint of them)
    const uint32_t* shell_start;   // [n + 1] same for the remaining tiles, after all head tiles
    const uint32_t* chunk_start;   // [n + 1] same for range chunks
    const uint32_t* sample_start;  // [n + 1] same for auto-tune samples
    uint32_t* queue;               // tile queue counter
    int n;
    uint32_t total_tiles, total_chunks, total_samples;
    uint32_t total_head;  // work items of the head tiles
    int A;
    int threads;
    int buffers;  // 1 or 2 (2 only when every field is staged by TMA)
    int num_sms;
};

cudaError_t launch_batch_prologue(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_batch_range_tune(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_batch_gather(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_batch_compress(const BatchLaunch& b, cudaStream_t st);
cudaError_t launch_batch_scatter(const BatchLaunch& b, uint32_t* status, uint32_t* queue, cudaStream_t st);
cudaError_t launch_decompress_batch(const BatchLaunch& b, uint32_t* status, uint32_t* queue, cudaStream_t st);

// Quantization-code reordering (Sec. 5.2.2, Eq. 3): per level l = 0..L, the
// stride-2^l grid's points along d1 and d2 (D), their halves rounded up (H)
// and the first sequence position of the level (prefix; the anchors, l = L,
// start at 0).
struct ReorderGeo {
    uint32_t n0, n1, n2;
    uint32_t segs;  // row segments per row
    int L;
    uint32_t D1[HI_MAX_LEVELS], D2[HI_MAX_LEVELS];
    uint32_t H1[HI_MAX_LEVELS], H2[HI_MAX_LEVELS];
    uint32_t prefix[HI_MAX_LEVELS];
};
ReorderGeo make_reorder_geo(const int64_t n[3], int L);
cudaError_t launch_reorder(const ReorderGeo& G, const uint8_t* src, uint8_t* dst, bool inverse, int num_sms,
                           cudaStream_t st);

// Throughput-mode lossless pipeline TCMS1-BIT1-RRE1 (Sec. 5.2.3).
size_t tp_ws_bytes(uint64_t n);
uint64_t tp_stream_bound(uint64_t n);
size_t cr_ws_bytes(uint64_t n);
uint64_t cr_stream_bound(uint64_t n);
cudaError_t launch_cr_encode(const uint8_t* in, uint64_t n, uint8_t* out, uint64_t* len, void* ws, int num_sms,
                             cudaStream_t st);
cudaError_t launch_cr_decode(const uint8_t* in, uint64_t in_len, uint64_t n, uint8_t* out, uint32_t* status,
                             void* ws, int num_sms, cudaStream_t st);
cudaError_t launch_tp_encode(const uint8_t* in, uint64_t n, uint8_t* out, uint64_t* len, void* ws, int num_sms,
                             cudaStream_t st);
cudaError_t launch_tp_decode(const uint8_t* in, uint64_t in_len, uint64_t n, uint8_t* out, uint32_t* status, void* ws,
                             int num_sms, cudaStream_t st);

}  // namespace hi
