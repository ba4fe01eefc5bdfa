// hi_api.cu -- the C ABI (include/hi.h): argument validation, geometry,
// workspace layout, TMA descriptors and the launch sequence of each call.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <mutex>
#include <new>
#include <vector>

#include <cudaTypedefs.h>

#include "hi_device.cuh"
#include "hi_internal.h"

namespace hi {
namespace {

struct Geometry {
    FieldGeo g;
    int A, L;
    uint64_t n_anchors;
    int ndim_active;
    int m, stride;  // auto-tune samples
    TuneCands cands;
};

int ilog2_pow2(uint32_t A)
{
    if (A < 2 || A > 32 || (A & (A - 1))) return -1;
    int l = 0;
    while ((1u << l) < A) ++l;
    return l;
}

// Candidates of one level (Sec. 5.1.3): cubic before linear; permutations of
// the active dims in lexicographic order with inactive dims appended.
TuneCands make_cands(const uint64_t dims[3], bool with_md)
{
    TuneCands tc{};
    int act[3], na = 0, ina[3], ni = 0;
    for (int d = 0; d < 3; ++d) (dims[d] > 1 ? act[na++] : ina[ni++]) = d;
    int perms[6][3];
    int np = 0;
    if (na == 0) {
        perms[0][0] = 0, perms[0][1] = 1, perms[0][2] = 2;
        np = 1;
    } else {
        int idx[3] = {0, 1, 2};
        // lexicographic permutations of idx[0..na)
        do {
            for (int k = 0; k < na; ++k) perms[np][k] = act[idx[k]];
            for (int k = 0; k < ni; ++k) perms[np][na + k] = ina[k];
            ++np;
            // next permutation over the first na entries
            int i = na - 2;
            while (i >= 0 && idx[i] > idx[i + 1]) --i;
            if (i < 0) break;
            int j = na - 1;
            while (idx[j] < idx[i]) --j;
            int t = idx[i];
            idx[i] = idx[j], idx[j] = t;
            for (int a = i + 1, b = na - 1; a < b; ++a, --b) t = idx[a], idx[a] = idx[b], idx[b] = t;
        } while (true);
    }
    tc.nperm = np;
    tc.ncfg = 2 * np;
    for (int sp = 0; sp < 2; ++sp)
        for (int i = 0; i < np; ++i) {
            const int c = sp * np + i;
            tc.interp[c] = (uint8_t)(sp == 0 ? HI_CUBIC : HI_LINEAR);
            for (int k = 0; k < 3; ++k) tc.order[c][k] = (uint8_t)perms[i][k];
        }
    if (with_md && na >= 2) {  // the multi-dimensional scheme, cubic before linear (order field: the first sequence)
        for (int sp = 0; sp < 2; ++sp) {
            const int c = tc.ncfg++;
            tc.interp[c] = (uint8_t)(sp == 0 ? HI_MD_CUBIC : HI_MD_LINEAR);
            for (int k = 0; k < 3; ++k) tc.order[c][k] = (uint8_t)perms[0][k];
        }
    }
    return tc;
}

hi_status make_geometry(const hi_params* p, Geometry* G)
{
    if (!p || (p->tuning & ~0xFu) != 0 || ((p->tuning >> 2) & 3u) == 3u || (p->tuning & 3u) == 3u) return HI_EINVAL;
    const int L = ilog2_pow2(p->anchor_stride);
    if (L < 0) return HI_EINVAL;
    if (!(p->eb > 0.0) || !std::isfinite(p->eb)) return HI_EINVAL;
    if (p->eb_mode != HI_EB_ABS && p->eb_mode != HI_EB_REL) return HI_EINVAL;
    if (p->autotune > 2) return HI_EINVAL;
    const int A = (int)p->anchor_stride;
    G->A = A;
    G->L = L;
    uint64_t N = 1, na_all = 1, nt = 1;
    int nact = 0;
    for (int d = 0; d < 3; ++d) {
        const uint64_t n = p->dims[d];
        if (n < 1 || n > 0x7fffffffull) return HI_EINVAL;
        N *= n;
        if (N >= (1ull << 32)) return HI_EINVAL;  // uint32 outlier indices
        G->g.n[d] = (int64_t)n;
        G->g.nb[d] = (n == 1) ? 1 : (int)((n - 1 + A - 1) / A);
        G->g.na[d] = (int)((n - 1) / A + 1);
        na_all *= (uint64_t)G->g.na[d];
        nt *= (uint64_t)G->g.nb[d];
        if (n > 1) ++nact;
    }
    if (nt > 0x7fffffffull) return HI_EINVAL;
    if (!p->autotune) {
        for (int l = 0; l < L; ++l) {
            const hi_level& lv = p->level[l];
            if (lv.interp > HI_MD_CUBIC) return HI_EINVAL;
            int seen = 0;
            for (int k = 0; k < 3; ++k) {
                if (lv.order[k] > 2) return HI_EINVAL;
                seen |= 1 << lv.order[k];
            }
            if (seen != 7) return HI_EINVAL;
        }
    }
    G->g.N = (int64_t)N;
    G->g.ntiles = (int)nt;
    // 3D fields: the tiles below the last block along every dim first in the
    // queue (whole tiles that own no upper face: the pipelined kernels' fast
    // tiles), then the last blocks, face by face
    for (int d = 0; d < 3; ++d) G->g.ni[d] = G->g.nb[d] - (nact == 3 ? 1 : 0);
    G->g.b0 = (p->dims[0] > 1) ? A + 1 : 1;
    G->n_anchors = na_all;
    G->ndim_active = nact;
    // auto-tune sample: 0.2% of the points in whole blocks, every (nt/m)-th block
    double vol = 1.0;
    for (int k = 0; k < nact; ++k) vol *= A;
    long long m = (long long)std::floor(0.002 * (double)N / vol + 0.5);
    if (m < 1) m = 1;
    if (m > (long long)nt) m = (long long)nt;
    G->m = (int)m;
    G->stride = (int)(nt / (uint64_t)m);
    G->cands = make_cands(p->dims, p->autotune == 2);
    return HI_OK;
}

constexpr size_t kWsTicket = 0;  // uint32: last-CTA ticket of the range pass
constexpr size_t kWsQueue = 4;   // uint32: tile queue of the predict / reconstruct kernels
constexpr size_t kWsTuneTicket = 8;  // uint32: last-CTA ticket of the auto-tuner (left at 0)
constexpr size_t kWsPartials = 256;
constexpr size_t kWsTune = kWsPartials + sizeof(float2) * kRangeBlocks;

size_t workspace_bytes(const Geometry& G)
{
    static_assert(kWsTune >= HI_DECOMPRESS_WS_BYTES, "workspace layout");
    return kWsTune + sizeof(double) * (size_t)G.m * G.L * (size_t)G.cands.ncfg;
}

PFN_cuTensorMapEncodeTiled_v12000 get_encode()
{
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
    });
    return fn;
}

// 3D box descriptor over a row-major [n0][n1][n2] array of elem-byte values;
// box = (bx, P, b0) elements, zero fill outside the field.
bool encode_box(CUtensorMap* map, const void* base, CUtensorMapDataType dt, int elem, const FieldGeo& g, int bx,
                int P)
{
    auto enc = get_encode();
    if (!enc) return false;
    if ((reinterpret_cast<uintptr_t>(base) & 15) != 0) return false;
    if (((uint64_t)g.n[2] * elem) % 16 != 0) return false;
    const cuuint64_t dims[3] = {(cuuint64_t)g.n[2], (cuuint64_t)g.n[1], (cuuint64_t)g.n[0]};
    const cuuint64_t strides[2] = {(cuuint64_t)g.n[2] * elem, (cuuint64_t)g.n[1] * g.n[2] * elem};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)P, (cuuint32_t)g.b0};
    const cuuint32_t es[3] = {1, 1, 1};
    CUresult r = enc(map, dt, 3, const_cast<void*>(base), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

template <int A>
struct PX_of {
    static constexpr int PX = TileGeom<A>::PX;
    static constexpr int CX = TileGeom<A>::CX;
};

void pitches(int A, int* PX, int* CX)
{
    switch (A) {
    case 2: *PX = PX_of<2>::PX, *CX = PX_of<2>::CX; break;
    case 4: *PX = PX_of<4>::PX, *CX = PX_of<4>::CX; break;
    case 8: *PX = PX_of<8>::PX, *CX = PX_of<8>::CX; break;
    case 16: *PX = PX_of<16>::PX, *CX = PX_of<16>::CX; break;
    default: *PX = PX_of<32>::PX, *CX = PX_of<32>::CX; break;
    }
}

constexpr int kMaxDevices = 64;

int num_sms()
{
    static std::mutex mu;
    static int cache[kMaxDevices] = {};
    int dev = 0, n = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 1;
    if (dev >= 0 && dev < kMaxDevices) {
        std::lock_guard<std::mutex> lock(mu);
        if (cache[dev] > 0) return cache[dev];
    }
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 1;
    if (n < 1) n = 1;
    if (dev >= 0 && dev < kMaxDevices) {
        std::lock_guard<std::mutex> lock(mu);
        cache[dev] = n;
    }
    return n;
}

int threads_for(const Geometry& G, uint32_t tuning)
{
    static const int kThreads[4] = {0, 64, 128, 128};
    if (tuning & 3u) return kThreads[tuning & 3u];
    // one tile per CTA: 128 threads keep the passes busy and let several tiles
    // share an SM (measured on GB300 for 17^3 tiles); small 1D/2D tiles use 64
    const long long vol = (long long)G.g.b0 * (G.A + 1) * ((G.g.n[1] > 1) ? (G.A + 1) : 1);
    if (vol >= 512) return 128;
    return 64;
}

// Workspace of hi_compress_static_ws: one fixed array per device, part of
// this library's device image, so that the call allocates nothing.
static __device__ __align__(256) unsigned char g_static_ws[HI_STATIC_WS_BYTES];

// The current context (driver API, through the runtime's entry-point query);
// nullptr when it cannot be had.
using PFN_ctx_get_current = CUresult (*)(CUcontext*);
CUcontext current_context()
{
    static PFN_ctx_get_current fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void* ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_ctx_get_current>(ptr);
    });
    CUcontext c = nullptr;
    if (!fn || fn(&c) != CUDA_SUCCESS) return nullptr;
    return c;
}

// Device address of g_static_ws on the current device, looked up once per
// device and context: a device reset (or a released and re-created primary
// context) gives a new context, and the address is looked up again; nullptr
// if the look-up fails.
void* static_ws_address()
{
    static std::mutex mu;
    static void* addr[kMaxDevices] = {};
    static CUcontext ctx[kMaxDevices] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    const CUcontext c = current_context();
    std::lock_guard<std::mutex> lock(mu);
    if (!addr[dev] || !c || ctx[dev] != c) {
        void* a = nullptr;
        if (cudaGetSymbolAddress(&a, g_static_ws) != cudaSuccess) return nullptr;
        addr[dev] = a;
        ctx[dev] = current_context();  // the look-up has made the device's context current
    }
    return addr[dev];
}

thread_local cudaEvent_t t_events[8];
thread_local bool t_events_on = false;

inline void stage_event(int k, cudaStream_t st)
{
    if (t_events_on) cudaEventRecord(t_events[k], st);
}

inline bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

hi_status cuda_status(cudaError_t e) { return e == cudaSuccess ? HI_OK : HI_ECUDA; }

}  // namespace
}  // namespace hi

using namespace hi;

extern "C" {

uint32_t hi_version(void) { return HI_VERSION; }

const char* hi_status_str(int s)
{
    switch (s) {
    case HI_OK: return "ok";
    case HI_EINVAL: return "invalid argument";
    case HI_ENOMEM: return "workspace too small";
    case HI_ECAPACITY: return "outlier capacity exceeded";
    case HI_ECUDA: return "CUDA error";
    case HI_ETIMEOUT: return "device wait timed out";
    case HI_ECORRUPT: return "corrupt compressed record";
    default: return "unknown status";
    }
}

hi_status hi_resolve_eps(uint32_t eb_mode, double eb, float vmin, float vmax, hi_eps* out)
{
    if (!out || (eb_mode != HI_EB_ABS && eb_mode != HI_EB_REL) || !(eb > 0.0) || !std::isfinite(eb))
        return HI_EINVAL;
    double eps = eb;
    if (eb_mode == HI_EB_REL) {
        const double range = (double)vmax - (double)vmin;
        if (range > 0.0) eps = eb * range;
    }
    const double two_eps = 2.0 * eps;
    float eb_f = (float)eps;  // round to nearest, then down to the largest float <= eps
    if ((double)eb_f > eps) eb_f = std::nextafter(eb_f, 0.0f);
    const float ebx2_f = (float)two_eps;
    const float r_f = (float)(1.0 / two_eps);
    if (!(eps > 0.0) || !std::isfinite(eps) || !(eb_f > 0.0f) || !std::isfinite(ebx2_f) || !(r_f > 0.0f) ||
        !std::isfinite(r_f))
        return HI_EINVAL;
    out->eps = eps;
    out->eb_f = eb_f;
    out->ebx2_f = ebx2_f;
    out->r_f = r_f;
    out->pad = 0.0f;
    return HI_OK;
}

hi_status hi_estimate_cr(const uint32_t* h_hist, uint64_t n_outliers, uint64_t n_anchors, uint64_t n_points,
                         uint64_t header_bytes, hi_cr_estimate* out)
{
    if (!h_hist || !out || n_points == 0) return HI_EINVAL;
    double total = 0.0;
    for (int k = 0; k < 256; ++k) total += (double)h_hist[k];
    double H = 0.0;
    if (total > 0.0)
        for (int k = 0; k < 256; ++k)
            if (h_hist[k] > 0) {
                const double q = (double)h_hist[k] / total;
                H -= q * std::log2(q);
            }
    const uint64_t nbytes =
        (uint64_t)std::ceil(total * H / 8.0) + 8 * n_outliers + 4 * n_anchors + header_bytes;
    out->entropy_bits = H;
    out->est_bytes = nbytes;
    out->cr = nbytes > 0 ? 4.0 * (double)n_points / (double)nbytes : INFINITY;
    out->bit_rate = 8.0 * (double)nbytes / (double)n_points;
    return HI_OK;
}

hi_status hi_query(const hi_params* p, uint64_t* n_points, uint64_t* n_anchors, uint64_t* n_blocks,
                   size_t* ws_bytes)
{
    Geometry G;
    const hi_status s = make_geometry(p, &G);
    if (s != HI_OK) return s;
    if (n_points) *n_points = (uint64_t)G.g.N;
    if (n_anchors) *n_anchors = G.n_anchors;
    if (n_blocks) *n_blocks = (uint64_t)G.g.ntiles;
    if (ws_bytes) *ws_bytes = workspace_bytes(G);
    return HI_OK;
}

static TuneLaunch tune_launch(const Geometry& G, const float* d_x, hi_header* d_header, void* d_ws)
{
    TuneLaunch t{};
    int PX, CX;
    pitches(G.A, &PX, &CX);
    t.use_tma = G.A >= 4 && encode_box(&t.tmap, d_x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, G.g, PX, G.A + 1);
    t.tma_bytes = (uint32_t)(PX * (G.A + 1) * G.g.b0 * 4);
    t.g = G.g;
    t.x = d_x;
    t.cands = G.cands;
    t.m = G.m;
    t.stride = G.stride;
    t.err = reinterpret_cast<double*>(static_cast<char*>(d_ws) + kWsTune);
    t.ticket = reinterpret_cast<uint32_t*>(static_cast<char*>(d_ws) + kWsTuneTicket);
    t.hdr = d_header;
    return t;
}

static hi_status enqueue_tune(const Geometry& G, const float* d_x, hi_header* d_header, void* d_ws,
                              cudaStream_t stream)
{
    return cuda_status(launch_tune(G.A, tune_launch(G, d_x, d_header, d_ws), stream));
}

// Whether the predict-quantize kernel can write the reordered sequence from
// its staged codes: A = 8 or 16, every tile row whole (n2 a multiple of A),
// the sequence 16-byte aligned with fewer than 2^32 places, and every run
// of a tile row (A >> l codes on level l, half of them for the odd columns
// of a row of even subgrid coordinates) starting at a multiple of its
// length: the terms of its place are multiples of A >> l.
static bool seq_fusable(const Geometry& G, const ReorderGeo& R, const uint8_t* d_seq)
{
    if ((G.A != 8 && G.A != 16) || G.g.n[2] % G.A != 0) return false;
    if (!aligned(d_seq, 16) || G.g.N >= (int64_t(1) << 32)) return false;
    for (int l = 0; l < G.L; ++l) {
        const uint64_t c = (uint64_t)(G.A >> l);
        if (R.prefix[l] % c || R.D2[l] % c || ((uint64_t)R.H1[l] * R.H2[l]) % c || R.H2[l] % c) return false;
    }
    return true;
}

static hi_status compress_impl(const hi_params* p, const float* d_x, uint8_t* d_codes, uint8_t* d_seq,
                               float* d_anchors, uint32_t* d_out_idx, float* d_out_val, uint64_t out_cap,
                               uint32_t* d_hist, float* d_recon, hi_header* d_header, void* d_ws, size_t ws_bytes,
                               cudaStream_t stream)
{
    Geometry G;
    hi_status s = make_geometry(p, &G);
    if (s != HI_OK) return s;
    if (!d_x || !d_codes || !d_anchors || !d_header || !d_ws) return HI_EINVAL;
    if (d_seq) {
        const uintptr_t a = reinterpret_cast<uintptr_t>(d_codes), b = reinterpret_cast<uintptr_t>(d_seq);
        const uintptr_t n = (uintptr_t)G.g.N;
        if (a < b + n && b < a + n) return HI_EINVAL;  // overlapping code arrays
    }
    if (out_cap > 0 && (!d_out_idx || !d_out_val)) return HI_EINVAL;
    if (!aligned(d_x, 4) || !aligned(d_ws, 8) || !aligned(d_header, 8)) return HI_EINVAL;
    if (ws_bytes < workspace_bytes(G)) return HI_ENOMEM;

    char* ws = static_cast<char*>(d_ws);
    uint32_t* ticket = reinterpret_cast<uint32_t*>(ws + kWsTicket);
    uint32_t* queue = reinterpret_cast<uint32_t*>(ws + kWsQueue);
    stage_event(0, stream);
    cudaError_t e =
        launch_prologue(d_header, *p, G.n_anchors, out_cap, (uint32_t)G.L, d_hist, ticket, queue, stream);
    if (e != cudaSuccess) return HI_ECUDA;
    stage_event(1, stream);
    if (p->eb_mode == HI_EB_REL && p->autotune) {
        // one launch: the auto-tuner's blocks run beside the range pass (independent of each other)
        int nb = kRangeBlocks;
        const int64_t need = (G.g.N + 2047) / 2048;
        if (need < nb) nb = (int)(need > 0 ? need : 1);
        e = launch_range_tune(G.A, tune_launch(G, d_x, d_header, d_ws), reinterpret_cast<float2*>(ws + kWsPartials),
                              nb, ticket, stream);
        if (e != cudaSuccess) return HI_ECUDA;
        stage_event(2, stream);
    } else {
        if (p->eb_mode == HI_EB_REL) {
            int nb = kRangeBlocks;
            const int64_t need = (G.g.N + 4095) / 4096;
            if (need < nb) nb = (int)(need > 0 ? need : 1);
            e = launch_range(d_x, G.g.N, reinterpret_cast<float2*>(ws + kWsPartials), nb, ticket, d_header,
                             stream);
            if (e != cudaSuccess) return HI_ECUDA;
        }
        stage_event(2, stream);
        if (p->autotune) {
            s = enqueue_tune(G, d_x, d_header, d_ws, stream);
            if (s != HI_OK) return s;
        }
    }
    stage_event(3, stream);
    CompressLaunch c{};
    int PX, CX;
    pitches(G.A, &PX, &CX);
    // a TMA box must start at an x coordinate whose byte offset is a multiple
    // of 16: tile origins are multiples of A, so floats need A >= 4
    const bool tma = G.A >= 4 && encode_box(&c.tmap, d_x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, G.g, PX, G.A + 1);
    c.g = G.g;
    c.x = d_x;
    c.codes = d_codes;
    c.anchors = d_anchors;
    c.out_idx = d_out_idx;
    c.out_val = d_out_val;
    c.out_cap = out_cap;
    c.hist = d_hist;
    c.recon = d_recon;
    c.hdr = d_header;
    c.queue = queue;
    c.tma_bytes = (uint32_t)(PX * (G.A + 1) * G.g.b0 * 4);
    const int ch = G.A >= 16 ? 16 : 8;
    c.flags = (tma ? kFlagTma : 0) |
              ((G.g.n[2] % ch == 0 && aligned(d_codes, 16)) ? kFlagVecCodes : 0);
    c.threads = threads_for(G, p->tuning);
    c.buffers = (int)((p->tuning >> 2) & 3u);
    c.num_sms = num_sms();
    c.max_ctas = 0;
    ReorderGeo R{};
    if (d_seq) {
        R = make_reorder_geo(G.g.n, G.L);
        if (seq_fusable(G, R, d_seq)) {
            c.seq = d_seq;
            for (int l = 0; l <= G.L; ++l) {
                c.sg.D1[l] = R.D1[l], c.sg.D2[l] = R.D2[l];
                c.sg.H12[l] = R.H1[l] * R.H2[l], c.sg.H2[l] = R.H2[l];
                c.sg.prefix[l] = R.prefix[l];
            }
        }
    }
    s = cuda_status(launch_compress(G.A, c, stream));
    stage_event(4, stream);
    if (s == HI_OK && d_seq && !c.seq) s = cuda_status(launch_reorder(R, d_codes, d_seq, false, num_sms(), stream));
    return s;
}

hi_status hi_compress(const hi_params* p, const float* d_x, uint8_t* d_codes, float* d_anchors,
                      uint32_t* d_out_idx, float* d_out_val, uint64_t out_cap, uint32_t* d_hist,
                      float* d_recon, hi_header* d_header, void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    return compress_impl(p, d_x, d_codes, nullptr, d_anchors, d_out_idx, d_out_val, out_cap, d_hist, d_recon,
                         d_header, d_ws, ws_bytes, stream);
}

hi_status hi_compress_seq(const hi_params* p, const float* d_x, uint8_t* d_codes, uint8_t* d_seq,
                          float* d_anchors, uint32_t* d_out_idx, float* d_out_val, uint64_t out_cap,
                          uint32_t* d_hist, float* d_recon, hi_header* d_header, void* d_ws, size_t ws_bytes,
                          cudaStream_t stream)
{
    if (!d_seq) return HI_EINVAL;
    return compress_impl(p, d_x, d_codes, d_seq, d_anchors, d_out_idx, d_out_val, out_cap, d_hist, d_recon,
                         d_header, d_ws, ws_bytes, stream);
}

int hi_compress_seq_fused(const hi_params* p, const uint8_t* d_codes, const uint8_t* d_seq)
{
    Geometry G;
    if (!p || !d_codes || make_geometry(p, &G) != HI_OK) return 0;
    return seq_fusable(G, make_reorder_geo(G.g.n, G.L), d_seq) ? 1 : 0;
}

hi_status hi_compress_static_ws(const hi_params* p, const float* d_x, uint8_t* d_codes, float* d_anchors,
                                uint32_t* d_out_idx, float* d_out_val, uint64_t out_cap, uint32_t* d_hist,
                                float* d_recon, hi_header* d_header, cudaStream_t stream)
{
    Geometry G;
    const hi_status s = make_geometry(p, &G);
    if (s != HI_OK) return s;
    if (workspace_bytes(G) > HI_STATIC_WS_BYTES) return HI_ENOMEM;
    void* ws = static_ws_address();
    if (!ws) return HI_ECUDA;
    return hi_compress(p, d_x, d_codes, d_anchors, d_out_idx, d_out_val, out_cap, d_hist, d_recon, d_header, ws,
                       HI_STATIC_WS_BYTES, stream);
}

hi_status hi_decompress(const hi_params* p, const hi_header* d_header, const uint8_t* d_codes,
                        const float* d_anchors, const uint32_t* d_out_idx, const float* d_out_val,
                        uint64_t out_cap, float* d_out, uint32_t* d_status, void* d_ws, size_t ws_bytes,
                        cudaStream_t stream)
{
    Geometry G;
    hi_params q = *p;
    q.autotune = 1;  // the level configuration comes from the header
    hi_status s = make_geometry(&q, &G);
    if (s != HI_OK) return s;
    if (!d_header || !d_codes || !d_anchors || !d_out) return HI_EINVAL;
    if (out_cap > 0 && (!d_out_idx || !d_out_val)) return HI_EINVAL;
    if (!aligned(d_out, 4) || !d_ws || !aligned(d_ws, 8)) return HI_EINVAL;
    if (ws_bytes < HI_DECOMPRESS_WS_BYTES) return HI_ENOMEM;
    uint32_t* queue = reinterpret_cast<uint32_t*>(static_cast<char*>(d_ws) + kWsQueue);
    cudaError_t e;
    stage_event(5, stream);
    if (d_status) {
        e = cudaMemsetAsync(d_status, 0, sizeof(uint32_t), stream);
        if (e != cudaSuccess) return HI_ECUDA;
    }
    e = launch_scatter(d_out_idx, d_out_val, out_cap, d_header, G.g.N, d_out, d_status, queue, stream);
    if (e != cudaSuccess) return HI_ECUDA;
    stage_event(6, stream);
    DecompressLaunch c{};
    int PX, CX;
    pitches(G.A, &PX, &CX);
    // byte-sized codes: the box origin x = t * A is 16-byte aligned only for A >= 16
    const bool tma = G.A >= 16 && encode_box(&c.cmap, d_codes, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, G.g, CX, G.A + 1);
    c.g = G.g;
    c.codes = d_codes;
    c.anchors = d_anchors;
    c.out = d_out;
    c.hdr = d_header;
    c.status = d_status;
    c.queue = queue;
    c.tma_bytes = (uint32_t)(CX * (G.A + 1) * G.g.b0);
    c.flags = (tma ? kFlagTma : 0) | ((G.g.n[2] % 4 == 0 && aligned(d_out, 16)) ? kFlagVecOut : 0);
    c.threads = threads_for(G, p->tuning);
    c.buffers = (int)((p->tuning >> 2) & 3u);
    c.num_sms = num_sms();
    c.max_ctas = 0;
    s = cuda_status(launch_decompress(G.A, c, stream));
    stage_event(7, stream);
    return s;
}

hi_status hi_autotune(const hi_params* p, const float* d_x, hi_header* d_header, void* d_ws, size_t ws_bytes,
                      cudaStream_t stream)
{
    Geometry G;
    hi_params q = *p;
    if (q.autotune == 0) q.autotune = 1;
    hi_status s = make_geometry(&q, &G);
    if (s != HI_OK) return s;
    if (!d_x || !d_header || !d_ws || !aligned(d_ws, 8)) return HI_EINVAL;
    if (ws_bytes < workspace_bytes(G)) return HI_ENOMEM;
    if (cudaMemsetAsync(static_cast<char*>(d_ws) + kWsTuneTicket, 0, sizeof(uint32_t), stream) != cudaSuccess)
        return HI_ECUDA;
    return enqueue_tune(G, d_x, d_header, d_ws, stream);
}

hi_status hi_autotune_select(const hi_params* p, const double* h_err, size_t h_err_len, hi_params* out)
{
    if (!p || !h_err || !out) return HI_EINVAL;
    Geometry G;
    hi_params q = *p;
    if (q.autotune == 0) q.autotune = 1;
    const hi_status s = make_geometry(&q, &G);
    if (s != HI_OK) return s;
    const int m = G.m, L = G.L, nc = G.cands.ncfg;
    if (h_err_len < (size_t)m * L * nc) return HI_EINVAL;
    for (int l = 0; l < L; ++l) {
        int best = 0;
        double best_sum = 0.0;
        for (int c = 0; c < nc; ++c) {
            double part[32];  // the device's lane partials, then its xor butterfly
            for (int j = 0; j < 32; ++j) {
                double a = 0.0;
                for (int k = j; k < m; k += 32) a += h_err[((size_t)k * L + l) * nc + c];
                part[j] = a;
            }
            for (int off = 16; off > 0; off >>= 1) {
                double nxt[32];
                for (int j = 0; j < 32; ++j) nxt[j] = part[j] + part[j ^ off];
                for (int j = 0; j < 32; ++j) part[j] = nxt[j];
            }
            if (c == 0 || part[0] < best_sum) best = c, best_sum = part[0];
        }
        out->level[l].interp = G.cands.interp[best];
        for (int k = 0; k < 3; ++k) out->level[l].order[k] = G.cands.order[best][k];
    }
    return HI_OK;
}

hi_status hi_autotune_errors(const hi_params* p, const void* d_ws, double* h_err, size_t h_err_len, uint32_t* m,
                             uint32_t* L, uint32_t* ncfg, cudaStream_t stream)
{
    Geometry G;
    hi_params q = *p;
    if (q.autotune == 0) q.autotune = 1;
    hi_status s = make_geometry(&q, &G);
    if (s != HI_OK) return s;
    if (m) *m = (uint32_t)G.m;
    if (L) *L = (uint32_t)G.L;
    if (ncfg) *ncfg = (uint32_t)G.cands.ncfg;
    const size_t n = (size_t)G.m * G.L * G.cands.ncfg;
    if (!h_err) return HI_OK;
    if (h_err_len < n || !d_ws) return HI_EINVAL;
    cudaError_t e = cudaMemcpyAsync(h_err, static_cast<const char*>(d_ws) + kWsTune, n * sizeof(double),
                                    cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return HI_ECUDA;
    return cuda_status(cudaStreamSynchronize(stream));
}

// ---------------------------------------------------------------------------
// Batches
// ---------------------------------------------------------------------------
static size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Geometry of every field and the workspace layout of the batch.
static hi_status batch_layout(uint32_t n, const hi_batch_field* f, std::vector<Geometry>* geo, hi_batch_plan* plan)
{
    if (n == 0 || !f || !plan) return HI_EINVAL;
    geo->resize(n);
    std::memset(plan, 0, sizeof(*plan));
    uint64_t tiles = 0, chunks = 0, samples = 0, err = 0;
    for (uint32_t i = 0; i < n; ++i) {
        Geometry& G = (*geo)[i];
        const hi_status s = make_geometry(&f[i].p, &G);
        if (s != HI_OK) return s;
        if (i == 0) plan->anchor_stride = f[i].p.anchor_stride;
        if (f[i].p.anchor_stride != plan->anchor_stride) return HI_EINVAL;
        tiles += (uint64_t)G.g.ntiles;
        if (f[i].p.eb_mode == HI_EB_REL) chunks += (uint64_t)((G.g.N + kBatchChunk - 1) / kBatchChunk);
        if (f[i].p.autotune) {
            samples += (uint64_t)G.m;
            err += (uint64_t)G.m * G.L * G.cands.ncfg;
        }
    }
    if (plan->anchor_stride != 8 && plan->anchor_stride != 16) return HI_EINVAL;
    if (tiles > 0x7fffffffull || chunks > 0x7fffffffull || samples > 0x7fffffffull) return HI_EINVAL;
    plan->n_fields = n;
    plan->total_tiles = tiles;
    plan->total_chunks = chunks;
    plan->total_samples = samples;
    plan->off_table = 256;
    plan->off_prefix = align256(plan->off_table + sizeof(BatchField) * n);
    plan->off_tickets = align256(plan->off_prefix + sizeof(uint32_t) * 4 * (n + 1));
    plan->off_partials = align256(plan->off_tickets + sizeof(uint32_t) * 2 * n);
    plan->off_err = align256(plan->off_partials + sizeof(float2) * chunks);
    plan->ws_bytes = align256(plan->off_err + sizeof(double) * err);
    return HI_OK;
}

// The plan keeps the number of head work items in its first reserved word.
static uint32_t pre_total_head(const hi_batch_plan* plan) { return (uint32_t)plan->reserved[0]; }

static BatchLaunch batch_launch(const hi_batch_plan* plan, void* d_ws)
{
    char* ws = static_cast<char*>(d_ws);
    const uint32_t n = plan->n_fields;
    BatchLaunch b{};
    b.fields = reinterpret_cast<const BatchField*>(ws + plan->off_table);
    const uint32_t* pre = reinterpret_cast<const uint32_t*>(ws + plan->off_prefix);
    b.tile_start = pre;
    b.chunk_start = pre + (n + 1);
    b.sample_start = pre + 2 * (n + 1);
    b.shell_start = pre + 3 * (n + 1);
    b.total_head = pre_total_head(plan);
    b.queue = reinterpret_cast<uint32_t*>(ws);
    b.n = (int)n;
    b.total_tiles = (uint32_t)plan->total_tiles;
    b.total_chunks = (uint32_t)plan->total_chunks;
    b.total_samples = (uint32_t)plan->total_samples;
    b.A = (int)plan->anchor_stride;
    const uint32_t th = plan->tuning & 3u, bu = (plan->tuning >> 2) & 3u;
    b.threads = th == 1 ? 64 : 128;
    b.buffers = (bu == 2 && plan->all_tma) ? 2 : 1;
    b.num_sms = num_sms();
    return b;
}

hi_status hi_batch_query(uint32_t n, const hi_batch_field* h_fields, size_t* ws_bytes)
{
    std::vector<Geometry> geo;
    hi_batch_plan plan;
    const hi_status s = batch_layout(n, h_fields, &geo, &plan);
    if (s != HI_OK) return s;
    if (ws_bytes) *ws_bytes = (size_t)plan.ws_bytes;
    return HI_OK;
}

hi_status hi_batch_prepare(uint32_t n, const hi_batch_field* h_fields, uint32_t tuning, void* d_ws,
                           size_t ws_bytes, hi_batch_plan* h_plan, cudaStream_t stream)
{
    if ((tuning & ~0xFu) != 0 || (tuning & 3u) == 3u || ((tuning >> 2) & 3u) == 3u) return HI_EINVAL;
    std::vector<Geometry> geo;
    hi_batch_plan plan;
    hi_status s = batch_layout(n, h_fields, &geo, &plan);
    if (s != HI_OK) return s;
    if (!d_ws || !aligned(d_ws, 256)) return HI_EINVAL;
    if (ws_bytes < plan.ws_bytes) return HI_ENOMEM;
    for (uint32_t i = 0; i < n; ++i) {
        const hi_batch_field& f = h_fields[i];
        if (!f.d_codes || !f.d_anchors || !f.d_header) return HI_EINVAL;
        if (f.out_cap > 0 && (!f.d_out_idx || !f.d_out_val)) return HI_EINVAL;
        if ((f.d_x && !aligned(f.d_x, 4)) || !aligned(f.d_header, 8) || (f.d_out && !aligned(f.d_out, 4)))
            return HI_EINVAL;
    }
    plan.tuning = tuning;
    char* ws = static_cast<char*>(d_ws);
    const size_t host_bytes = plan.off_err;  // table, prefixes and tickets (partials / sums need no init)
    // host image of the table, aligned like the device copy
    const size_t host_alloc = align256(host_bytes);
    std::unique_ptr<unsigned char, void (*)(void*)> host(static_cast<unsigned char*>(std::aligned_alloc(256, host_alloc)),
                                                         std::free);
    if (!host) return HI_ENOMEM;
    std::memset(host.get(), 0, host_alloc);
    BatchField* table = reinterpret_cast<BatchField*>(host.get() + plan.off_table);
    uint32_t* pre = reinterpret_cast<uint32_t*>(host.get() + plan.off_prefix);
    uint32_t *ts = pre, *cs = pre + (n + 1), *ss = pre + 2 * (n + 1), *hs = pre + 3 * (n + 1);
    uint64_t tiles = 0, chunks = 0, samples = 0, err = 0, head = 0, shell = 0;
    bool all_tma = true, all_in = true, all_out = true;
    int PX, CX;
    pitches((int)plan.anchor_stride, &PX, &CX);
    for (uint32_t i = 0; i < n; ++i) {
        const hi_batch_field& f = h_fields[i];
        const Geometry& G = geo[i];
        BatchField& B = table[i];
        new (&B) BatchField();
        const bool tma = f.d_x && encode_box(&B.tmap, f.d_x, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, G.g, PX, G.A + 1);
        all_tma = all_tma && tma;
        all_in = all_in && f.d_x != nullptr;
        all_out = all_out && f.d_out != nullptr;
        // code boxes for the batched reconstruction (byte-sized: box origins are 16-byte aligned only for A >= 16)
        const bool ctma = G.A >= 16 && encode_box(&B.cmap, f.d_codes, CU_TENSOR_MAP_DATA_TYPE_UINT8, 1, G.g, CX, G.A + 1);
        B.out = f.d_out;
        B.ctma_bytes = (uint32_t)(CX * (G.A + 1) * G.g.b0);
        B.dflags = (ctma ? kFlagTma : 0) | ((G.g.n[2] % 4 == 0 && f.d_out && aligned(f.d_out, 16)) ? kFlagVecOut : 0);
        B.g = G.g;
        B.p = f.p;
        B.x = f.d_x;
        B.codes = f.d_codes;
        B.anchors = f.d_anchors;
        B.out_idx = f.d_out_idx;
        B.out_val = f.d_out_val;
        B.out_cap = f.out_cap;
        B.hist = f.d_hist;
        B.recon = f.d_recon;
        B.hdr = f.d_header;
        B.n_anchors = G.n_anchors;
        B.cands = G.cands;
        B.n_levels = (uint32_t)G.L;
        B.tma_bytes = (uint32_t)(PX * (G.A + 1) * G.g.b0 * 4);
        const int ch = G.A >= 16 ? 16 : 8;
        B.flags = (tma ? kFlagTma : 0) | ((G.g.n[2] % ch == 0 && aligned(f.d_codes, 16)) ? kFlagVecCodes : 0);
        B.cur.out = CompressOut{f.d_codes, f.d_anchors, f.d_out_idx, f.d_out_val, f.out_cap, f.d_recon, f.d_header,
                                (B.flags & kFlagVecCodes) != 0, f.d_hist != nullptr};
        B.cur.g = G.g;
        B.cur.x = f.d_x;
        B.cur.hist = f.d_hist;
        B.cur.flags = B.flags;
        B.m = f.p.autotune ? G.m : 0;
        B.stride = G.stride;
        B.nchunks = f.p.eb_mode == HI_EB_REL ? (uint32_t)((G.g.N + kBatchChunk - 1) / kBatchChunk) : 0u;
        B.partials = reinterpret_cast<float2*>(ws + plan.off_partials) + chunks;
        B.err = reinterpret_cast<double*>(ws + plan.off_err) + err;
        B.tickets = reinterpret_cast<uint32_t*>(ws + plan.off_tickets) + 2 * i;
        B.nint = (uint32_t)G.g.ni[0] * (uint32_t)G.g.ni[1] * (uint32_t)G.g.ni[2];
        ts[i] = (uint32_t)head;
        hs[i] = (uint32_t)shell;
        head += B.nint;
        shell += (uint64_t)G.g.ntiles - B.nint;
        cs[i] = (uint32_t)chunks;
        ss[i] = (uint32_t)samples;
        tiles += (uint64_t)G.g.ntiles;
        chunks += B.nchunks;
        samples += (uint64_t)B.m;
        err += (uint64_t)B.m * G.L * G.cands.ncfg;
    }
    ts[n] = (uint32_t)head;
    hs[n] = (uint32_t)shell;
    cs[n] = (uint32_t)chunks;
    ss[n] = (uint32_t)samples;
    plan.all_tma = all_tma ? 1u : 0u;
    plan.reserved[0] = head;
    plan.reserved[1] = (all_in ? 1u : 0u) | (all_out ? 2u : 0u);  // every field has an input / an output
    cudaError_t e = cudaMemcpyAsync(ws, host.get(), host_bytes, cudaMemcpyHostToDevice, stream);
    if (e != cudaSuccess) return HI_ECUDA;
    e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return HI_ECUDA;
    *h_plan = plan;
    return HI_OK;
}

hi_status hi_compress_batch(const hi_batch_plan* h_plan, void* d_ws, cudaStream_t stream)
{
    if (!h_plan || !d_ws || h_plan->n_fields == 0 || !(h_plan->reserved[1] & 1u)) return HI_EINVAL;
    const BatchLaunch b = batch_launch(h_plan, d_ws);
    stage_event(0, stream);
    if (launch_batch_prologue(b, stream) != cudaSuccess) return HI_ECUDA;
    stage_event(1, stream);
    if (launch_batch_range_tune(b, stream) != cudaSuccess) return HI_ECUDA;
    stage_event(2, stream);
    if (launch_batch_gather(b, stream) != cudaSuccess) return HI_ECUDA;
    stage_event(3, stream);
    const hi_status s = cuda_status(launch_batch_compress(b, stream));
    stage_event(4, stream);
    return s;
}

hi_status hi_decompress_batch(const hi_batch_plan* h_plan, void* d_ws, uint32_t* d_status, cudaStream_t stream)
{
    if (!h_plan || !d_ws || h_plan->n_fields == 0 || !(h_plan->reserved[1] & 2u)) return HI_EINVAL;
    if (d_status && !aligned(d_status, 4)) return HI_EINVAL;
    const BatchLaunch b = batch_launch(h_plan, d_ws);
    uint32_t* queue = reinterpret_cast<uint32_t*>(d_ws) + 1;  // the reconstruction's own counter
    if (d_status && cudaMemsetAsync(d_status, 0, sizeof(uint32_t), stream) != cudaSuccess) return HI_ECUDA;
    if (launch_batch_scatter(b, d_status, queue, stream) != cudaSuccess) return HI_ECUDA;
    return cuda_status(launch_decompress_batch(b, d_status, queue, stream));
}

hi_status hi_batch_tune_launch(hi_batch_plan* h_plan, void* d_ws, uint32_t reps, float* h_ms, cudaStream_t stream)
{
    if (!h_plan || !d_ws || reps == 0) return HI_EINVAL;
    static const uint32_t kCand[4] = {2u | (1u << 2), 1u | (1u << 2), 2u | (2u << 2), 1u | (2u << 2)};
    const uint32_t keep = h_plan->tuning;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return HI_ECUDA;
    }
    hi_status s = HI_OK;
    float best = 0.0f;
    uint32_t best_t = keep;
    for (int c = 0; c < 4 && s == HI_OK; ++c) {
        if (h_ms) h_ms[c] = 0.0f;
        if (((kCand[c] >> 2) & 3u) == 2u && !h_plan->all_tma) continue;
        h_plan->tuning = kCand[c];
        s = hi_compress_batch(h_plan, d_ws, stream);  // warm-up
        if (s != HI_OK) break;
        if (cudaEventRecord(e0, stream) != cudaSuccess) s = HI_ECUDA;
        for (uint32_t r = 0; r < reps && s == HI_OK; ++r) s = hi_compress_batch(h_plan, d_ws, stream);
        if (s != HI_OK) break;
        float ms = 0.0f;
        if (cudaEventRecord(e1, stream) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
            s = HI_ECUDA;
            break;
        }
        ms /= (float)reps;
        if (h_ms) h_ms[c] = ms;
        if (best == 0.0f || ms < best) best = ms, best_t = kCand[c];
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    h_plan->tuning = (s == HI_OK) ? best_t : keep;
    return s;
}

hi_status hi_set_stage_events(void* const* events, uint32_t n)
{
    if (!events) {
        t_events_on = false;
        return HI_OK;
    }
    if (n != 8) return HI_EINVAL;
    for (int k = 0; k < 8; ++k) {
        if (!events[k]) return HI_EINVAL;
        t_events[k] = static_cast<cudaEvent_t>(events[k]);
    }
    t_events_on = true;
    return HI_OK;
}

static hi_status reorder_call(const hi_params* p, const uint8_t* src, uint8_t* dst, bool inverse,
                              cudaStream_t stream)
{
    Geometry G;
    if (!p || !src || !dst) return HI_EINVAL;
    hi_status s = make_geometry(p, &G);
    if (s != HI_OK) return s;
    const uintptr_t a = reinterpret_cast<uintptr_t>(src), b = reinterpret_cast<uintptr_t>(dst);
    const uintptr_t n = (uintptr_t)G.g.N;
    if (a < b + n && b < a + n) return HI_EINVAL;  // overlapping buffers
    const ReorderGeo R = make_reorder_geo(G.g.n, G.L);
    return cuda_status(launch_reorder(R, src, dst, inverse, num_sms(), stream));
}

hi_status hi_reorder_codes(const hi_params* p, const uint8_t* d_codes, uint8_t* d_seq, cudaStream_t stream)
{
    return reorder_call(p, d_codes, d_seq, false, stream);
}

hi_status hi_unreorder_codes(const hi_params* p, const uint8_t* d_seq, uint8_t* d_codes, cudaStream_t stream)
{
    return reorder_call(p, d_seq, d_codes, true, stream);
}

hi_status hi_value_range(const hi_params* p, const float* d_x, hi_header* d_header, void* d_ws, size_t ws_bytes,
                         cudaStream_t stream)
{
    Geometry G;
    hi_status s = make_geometry(p, &G);
    if (s != HI_OK) return s;
    if (p->eb_mode != HI_EB_REL || !d_x || !d_header || !d_ws) return HI_EINVAL;
    if (!aligned(d_x, 4) || !aligned(d_ws, 8) || !aligned(d_header, 8)) return HI_EINVAL;
    if (ws_bytes < kWsTune) return HI_ENOMEM;
    char* ws = static_cast<char*>(d_ws);
    uint32_t* ticket = reinterpret_cast<uint32_t*>(ws + kWsTicket);
    uint32_t* queue = reinterpret_cast<uint32_t*>(ws + kWsQueue);
    cudaError_t e = launch_prologue(d_header, *p, G.n_anchors, 0, (uint32_t)G.L, nullptr, ticket, queue, stream);
    if (e != cudaSuccess) return HI_ECUDA;
    int nb = kRangeBlocks;
    const int64_t need = (G.g.N + 4095) / 4096;
    if (need < nb) nb = (int)(need > 0 ? need : 1);
    return cuda_status(
        launch_range(d_x, G.g.N, reinterpret_cast<float2*>(ws + kWsPartials), nb, ticket, d_header, stream));
}

hi_status hi_tp_query(uint64_t n, uint64_t* max_stream_bytes, size_t* ws_bytes)
{
    if (n >= (1ull << 44)) return HI_EINVAL;
    if (max_stream_bytes) *max_stream_bytes = tp_stream_bound(n);
    if (ws_bytes) *ws_bytes = tp_ws_bytes(n);
    return HI_OK;
}

hi_status hi_tp_encode(const uint8_t* d_in, uint64_t n, uint8_t* d_out, uint64_t out_cap, uint64_t* d_len,
                       void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (n >= (1ull << 44) || (n && !d_in) || !d_out || !d_len || !d_ws) return HI_EINVAL;
    if (!aligned(d_out, 16) || !aligned(d_len, 8) || !aligned(d_ws, 16)) return HI_EINVAL;
    if (out_cap < tp_stream_bound(n) || ws_bytes < tp_ws_bytes(n)) return HI_EINVAL;
    const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
    if (n && a < b + out_cap && b < a + n) return HI_EINVAL;
    return cuda_status(launch_tp_encode(d_in, n, d_out, d_len, d_ws, num_sms(), stream));
}

hi_status hi_tp_decode(const uint8_t* d_in, uint64_t in_len, uint8_t* d_out, uint64_t n, uint32_t* d_status,
                       void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (n >= (1ull << 44) || !d_in || (n && !d_out) || !d_ws) return HI_EINVAL;
    if (!aligned(d_in, 16) || !aligned(d_ws, 16) || (d_status && !aligned(d_status, 4))) return HI_EINVAL;
    const uint64_t nc = (n + 16383) / 16384;
    if (in_len < (16 + 4 * nc + 15) / 16 * 16 || ws_bytes < 8 * nc) return HI_EINVAL;
    return cuda_status(launch_tp_decode(d_in, in_len, n, d_out, d_status, d_ws, num_sms(), stream));
}

hi_status hi_cr_query(uint64_t n, uint64_t* max_stream_bytes, size_t* ws_bytes)
{
    if (n >= (1ull << 32)) return HI_EINVAL;
    if (max_stream_bytes) *max_stream_bytes = cr_stream_bound(n);
    if (ws_bytes) *ws_bytes = cr_ws_bytes(n);
    return HI_OK;
}

hi_status hi_cr_encode(const uint8_t* d_in, uint64_t n, uint8_t* d_out, uint64_t out_cap, uint64_t* d_len,
                       void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (n >= (1ull << 32) || (n && !d_in) || !d_out || !d_len || !d_ws) return HI_EINVAL;
    if ((n && !aligned(d_in, 16)) || !aligned(d_out, 16) || !aligned(d_len, 8) || !aligned(d_ws, 16)) return HI_EINVAL;
    if (out_cap < cr_stream_bound(n) || ws_bytes < cr_ws_bytes(n)) return HI_EINVAL;
    const uintptr_t a = reinterpret_cast<uintptr_t>(d_in), b = reinterpret_cast<uintptr_t>(d_out);
    if (n && a < b + out_cap && b < a + n) return HI_EINVAL;
    return cuda_status(launch_cr_encode(d_in, n, d_out, d_len, d_ws, num_sms(), stream));
}

hi_status hi_cr_decode(const uint8_t* d_in, uint64_t in_len, uint8_t* d_out, uint64_t n, uint32_t* d_status,
                       void* d_ws, size_t ws_bytes, cudaStream_t stream)
{
    if (n >= (1ull << 32) || !d_in || (n && !d_out) || !d_ws) return HI_EINVAL;
    if (!aligned(d_in, 16) || (n && !aligned(d_out, 16)) || !aligned(d_ws, 16) ||
        (d_status && !aligned(d_status, 4)))
        return HI_EINVAL;
    const uint64_t nb = (n + 4095) / 4096;
    if (in_len < (288 + 4 * nb + 15) / 16 * 16 || ws_bytes < cr_ws_bytes(n)) return HI_EINVAL;
    return cuda_status(launch_cr_decode(d_in, in_len, n, d_out, d_status, d_ws, num_sms(), stream));
}

hi_status hi_header_read(const hi_header* d_header, hi_header* h_header, cudaStream_t stream)
{
    if (!d_header || !h_header) return HI_EINVAL;
    cudaError_t e = cudaMemcpyAsync(h_header, d_header, sizeof(hi_header), cudaMemcpyDeviceToHost, stream);
    if (e != cudaSuccess) return HI_ECUDA;
    return cuda_status(cudaStreamSynchronize(stream));
}

}  // extern "C"

static_assert(sizeof(hi_header) == 168, "hi_header layout");
static_assert(sizeof(hi_params) == 80, "hi_params layout");
static_assert(sizeof(hi_batch_field) == 160, "hi_batch_field layout");
static_assert(sizeof(hi_batch_plan) == 120, "hi_batch_plan layout");
static_assert(sizeof(hi::BatchField) % 128 == 0, "field records stay 128-byte aligned");
