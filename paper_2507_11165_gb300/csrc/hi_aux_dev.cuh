// hi_aux_dev.cuh -- device functions of the stages around predict/quantize,
// shared by the single-field kernels (hi_aux.cu) and the batched ones
// (hi_batch.cu): the float32 quantizer constants (Eq. 1), header set-up, the
// value range for the value-range-relative bound (Sec. 6.1.4) and one block
// of the auto-tuner (Sec. 5.1.3).
#pragma once

#include <cstdint>

#include "hi_device.cuh"
#include "hi_internal.h"

namespace hi {

// eps and the float32 constants the quantizer uses (device, IEEE double):
//   eps = eb (absolute) or eb * (vmax - vmin) (relative; eb if the range is 0);
//   eb_f = eps rounded toward zero (the largest float <= eps),
//   ebx2_f = fl(2 eps), r_f = fl(1 / (2 eps)).
__device__ __forceinline__ void finalize_eps(hi_header* h, float vmin, float vmax)
{
    double eps;
    if (h->eb_mode == HI_EB_ABS) {
        eps = h->eb;
    } else {
        const double range = __dsub_rn((double)vmax, (double)vmin);
        eps = (range > 0.0) ? __dmul_rn(h->eb, range) : h->eb;
    }
    const double two_eps = __dmul_rn(2.0, eps);
    const float eb_f = __double2float_rz(eps);
    const float ebx2_f = __double2float_rn(two_eps);
    const float r_f = __double2float_rn(__ddiv_rn(1.0, two_eps));
    h->eps = eps;
    h->eb_f = eb_f;
    h->ebx2_f = ebx2_f;
    h->r_f = r_f;
    h->vmin = vmin;
    h->vmax = vmax;
    const bool ok = (eps > 0.0) && (eps < INFINITY) && (eb_f > 0.0f) && (fabsf(ebx2_f) < INFINITY) &&
                    (r_f > 0.0f) && (r_f < INFINITY);
    if (!ok) set_status(&h->status, HI_EINVAL);
}

// Header set-up of one compression (thread 0 writes the header; the CTA
// clears the histogram).  ticket_range, ticket_tune and queue may be NULL.
__device__ __forceinline__ void prologue_fill(hi_header* hdr, const hi_params& p, uint64_t n_anchors,
                                              uint64_t out_cap, uint32_t n_levels, uint32_t* hist,
                                              uint32_t* ticket_range, uint32_t* ticket_tune, uint32_t* queue)
{
    const int tid = threadIdx.x;
    if (hist)
        for (int i = tid; i < 256; i += blockDim.x) hist[i] = 0;
    if (tid == 0) {
        hdr->magic = HI_MAGIC;
        hdr->version = HI_VERSION;
        for (int d = 0; d < 3; ++d) hdr->dims[d] = p.dims[d];
        hdr->anchor_stride = p.anchor_stride;
        hdr->eb_mode = p.eb_mode;
        hdr->eb = p.eb;
        hdr->status = 0;
        hdr->n_outliers = 0;
        hdr->out_cap = out_cap;
        hdr->n_anchors = n_anchors;
        hdr->n_levels = n_levels;
        for (int l = 0; l < HI_MAX_LEVELS; ++l) hdr->level[l] = p.level[l];
        for (int k = 0; k < 7; ++k) hdr->reserved[k] = 0;
        if (ticket_range) *ticket_range = 0;
        if (ticket_tune) *ticket_tune = 0;
        if (queue) *queue = 0;
        if (p.eb_mode == HI_EB_ABS) finalize_eps(hdr, 0.0f, 0.0f);
    }
}

// A finite value (NaN and +-Inf are left out of the range).
__device__ __forceinline__ bool finite_f(float v) { return fabsf(v) < INFINITY; }

__device__ __forceinline__ void minmax4(const float4 f, float& mn, float& mx)
{
    if (finite_f(f.x)) mn = fminf(mn, f.x), mx = fmaxf(mx, f.x);
    if (finite_f(f.y)) mn = fminf(mn, f.y), mx = fmaxf(mx, f.y);
    if (finite_f(f.z)) mn = fminf(mn, f.z), mx = fmaxf(mx, f.z);
    if (finite_f(f.w)) mn = fminf(mn, f.w), mx = fmaxf(mx, f.w);
}

// Min and max over the finite values of x[lo, hi) that this thread visits:
// entries t0, t0 + stride, ... (in 16-byte vectors when x + lo is aligned,
// four loads in flight per thread).
__device__ __forceinline__ void range_accum(const float* __restrict__ x, int64_t lo, int64_t hi, int64_t t0,
                                            int64_t stride, float& mn, float& mx)
{
    const float* xs = x + lo;
    const int64_t n = hi - lo;
    int64_t head = 0;
    if ((reinterpret_cast<uintptr_t>(xs) & 15) == 0) {
        const int64_t n4 = n / 4;
        const float4* x4 = reinterpret_cast<const float4*>(xs);
        int64_t i = t0;
        for (; i + 3 * stride < n4; i += 4 * stride) {
            float4 f[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) f[u] = __ldcs(x4 + i + u * stride);
#pragma unroll
            for (int u = 0; u < 4; ++u) minmax4(f[u], mn, mx);
        }
        for (; i < n4; i += stride) minmax4(__ldcs(x4 + i), mn, mx);
        head = n4 * 4;
    }
    for (int64_t i = head + t0; i < n; i += stride) {
        const float f = xs[i];
        if (finite_f(f)) mn = fminf(mn, f), mx = fmaxf(mx, f);
    }
}

// CTA-wide min / max (exact in any order); the result is valid in thread 0.
__device__ __forceinline__ void block_minmax(float& mn, float& mx, float* s_mn, float* s_mx)
{
    for (int o = 16; o > 0; o >>= 1) {
        mn = fminf(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (lane == 0) s_mn[warp] = mn, s_mx[warp] = mx;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int w = 1; w < nw; ++w) mn = fminf(mn, s_mn[w]), mx = fmaxf(mx, s_mx[w]);
}

// The last CTA of a range pass: folds the nparts partials (min, max), reports
// a signed zero as +0 and a range with no finite value as [0, 0], and derives
// eps into hdr (all threads call it).
__device__ __forceinline__ void range_fold(const float2* partials, uint32_t nparts, hi_header* hdr, float* s_mn,
                                           float* s_mx)
{
    float mn = INFINITY, mx = -INFINITY;
    for (unsigned k = threadIdx.x; k < nparts; k += blockDim.x) {
        const float2 pk = __ldcg(partials + k);
        mn = fminf(mn, pk.x);
        mx = fmaxf(mx, pk.y);
    }
    __syncthreads();  // s_mn / s_mx may still be read from an earlier fold
    block_minmax(mn, mx, s_mn, s_mx);
    if (threadIdx.x == 0) {
        float a = mn, b = mx;
        if (!(a <= b)) a = 0.0f, b = 0.0f;
        a = __fadd_rn(a, 0.0f);
        b = __fadd_rn(b, 0.0f);
        finalize_eps(hdr, a, b);
    }
}

// One CTA `rb` of `nb` of a value-range pass over x[0, N): grid-strided
// streaming read, its partial (min, max) to partials[rb]; the last CTA to
// finish (ticket) folds the partials and derives eps into hdr.
__device__ __forceinline__ void range_block(const float* __restrict__ x, int64_t N, float2* partials, int rb,
                                            int nb, uint32_t* ticket, hi_header* hdr)
{
    __shared__ float s_mn[32], s_mx[32];
    __shared__ bool s_last;
    float mn = INFINITY, mx = -INFINITY;
    range_accum(x, 0, N, (int64_t)rb * blockDim.x + threadIdx.x, (int64_t)nb * blockDim.x, mn, mx);
    block_minmax(mn, mx, s_mn, s_mx);
    if (threadIdx.x == 0) {
        partials[rb] = make_float2(mn, mx);
        __threadfence();
        s_last = atomicAdd(ticket, 1u) == (uint32_t)nb - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    range_fold(partials, nb, hdr, s_mn, s_mx);
    if (threadIdx.x == 0) *ticket = 0;
}

// ---------------------------------------------------------------------------
// Auto-tune: a CTA (sample, candidate) computes, for every level, the sum of
// |x - p| over that level's points of its sampled block, with every
// prediction taken from the original values (no quantization), in the
// candidate's pass order.  Each term is a float, summed in double: per line
// into independent per-point accumulators (no long FP64 dependency chain),
// then over the block in a fixed order, so the sums are deterministic run to
// run.
// ---------------------------------------------------------------------------
template <int A, int S>
__device__ __forceinline__ double tune_pass(const float* __restrict__ v, bool cubic, int d, int stq, int str,
                                            const int e[3])
{
    using TG = TileGeom<A>;
    constexpr int NDM = A / (2 * S);
    const int q = (d == 0) ? 1 : 0, r = (d == 2) ? 1 : 2;
    const int ed = d == 0 ? e[0] : (d == 1 ? e[1] : e[2]);
    const int eq = q == 0 ? e[0] : e[1], er = r == 1 ? e[1] : e[2];
    if (ed < S) return 0.0;
    const int nd = (ed - S) / (2 * S) + 1;
    const int nq = eq / stq + 1, nr = er / str + 1;
    const int vpd = (d == 0 ? TG::PY : (d == 1 ? TG::PX : 1)) * S;
    const int vpq = q == 0 ? TG::PY : TG::PX, vpr = r == 1 ? TG::PX : 1;
    double acc = 0.0;
    for (int line = threadIdx.x; line < nq * nr; line += blockDim.x) {
        const int jq = line / nr, jr = line - jq * nr;
        const int vb = jq * stq * vpq + jr * str * vpr;
        float f[NDM + 1];
#pragma unroll
        for (int m = 0; m <= NDM; ++m) f[m] = (2 * m * S <= ed) ? v[vb + 2 * m * vpd] : 0.0f;
        double part[NDM];
#pragma unroll
        for (int k = 0; k < NDM; ++k) {
            part[k] = 0.0;
            if (k < nd) {
                const int c = (2 * k + 1) * S;
                const bool have_r = c + S <= ed, have_r3 = c + 3 * S <= ed;
                const float pr = predict(cubic, k >= 1, have_r, have_r3, k >= 1 ? f[k - 1] : 0.0f, f[k],
                                         have_r ? f[k + 1] : 0.0f, (k + 2 <= NDM && have_r3) ? f[k + 2] : 0.0f);
                part[k] = (double)fabsf(__fsub_rn(v[vb + (2 * k + 1) * vpd], pr));
            }
        }
#pragma unroll
        for (int k = 0; k < NDM; ++k) acc += part[k];
    }
    return acc;
}

// Open-loop error of the multi-dimensional scheme at stride S (the same
// phases and means as level_md, predictions from the original values).
template <int A>
__device__ __noinline__ double tune_md(const float* __restrict__ v, int S, bool cubic, const int e0, const int e1,
                                       const int e2)
{
    using TG = TileGeom<A>;
    const int e[3] = {e0, e1, e2};
    const int act = (e0 > 0 ? 1 : 0) | (e1 > 0 ? 2 : 0) | (e2 > 0 ? 4 : 0);
    double acc = 0.0;
    for (int m = 1; m < 8; ++m) {
        if (m & ~act) continue;
        int n[3];
#pragma unroll
        for (int d = 0; d < 3; ++d)
            n[d] = ((m >> d) & 1) ? (e[d] >= S ? (e[d] - S) / (2 * S) + 1 : 0) : e[d] / (2 * S) + 1;
        const int total = n[0] * n[1] * n[2];
        for (int i = threadIdx.x; i < total; i += blockDim.x) {
            const int j2 = i % n[2], r = i / n[2];
            const int j1 = r % n[1], j0 = r / n[1];
            const int jj[3] = {j0, j1, j2};
            int c[3];
#pragma unroll
            for (int d = 0; d < 3; ++d) c[d] = ((m >> d) & 1) ? (2 * jj[d] + 1) * S : 2 * jj[d] * S;
            const int vi = c[0] * TG::PY + c[1] * TG::PX + c[2];
            float p[3];
            int o[3];
            int best = -1;
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                p[d] = 0.0f;
                o[d] = -1;
                if (!((m >> d) & 1)) continue;
                const int st = (d == 0 ? TG::PY : (d == 1 ? TG::PX : 1)) * S;
                const bool have_r = c[d] + S <= e[d], have_l3 = c[d] >= 3 * S, have_r3 = c[d] + 3 * S <= e[d];
                const float b = v[vi - st];
                const float u = have_r ? v[vi + st] : 0.0f;
                const float a = have_l3 ? v[vi - 3 * st] : 0.0f;
                const float w = have_r3 ? v[vi + 3 * st] : 0.0f;
                p[d] = predict(cubic, have_l3, have_r, have_r3, a, b, u, w);
                o[d] = !have_r ? (have_l3 ? 1 : 0) : (!cubic ? 1 : ((have_l3 && have_r3) ? 3 : ((have_l3 || have_r3) ? 2 : 1)));
                best = o[d] > best ? o[d] : best;
            }
            float sum = 0.0f;
            int cnt = 0;
#pragma unroll
            for (int d = 0; d < 3; ++d)
                if (o[d] == best) {
                    sum = cnt == 0 ? p[d] : __fadd_rn(sum, p[d]);
                    ++cnt;
                }
            const float pr = cnt == 1 ? sum : (cnt == 2 ? __fmul_rn(sum, 0.5f) : __fdiv_rn(sum, 3.0f));
            acc += (double)fabsf(__fsub_rn(v[vi], pr));
        }
    }
    return acc;
}

template <int A, int LV>
__device__ __forceinline__ void tune_levels(const float* v, const hi_level& lv, const int e[3], double* acc)
{
    constexpr int S = 1 << LV;
    if (lv.interp == HI_MD_LINEAR || lv.interp == HI_MD_CUBIC) {
        acc[LV] = tune_md<A>(v, S, lv.interp == HI_MD_CUBIC, e[0], e[1], e[2]);
        if constexpr (LV > 0) tune_levels<A, LV - 1>(v, lv, e, acc);
        return;
    }
    const bool cubic = lv.interp == HI_CUBIC;
    double a = 0.0;
#pragma unroll
    for (int p = 0; p < 3; ++p) {
        const int d = lv.order[p];
        const int q = (d == 0) ? 1 : 0, r = (d == 2) ? 1 : 2;
        const int posq = (lv.order[0] == q) ? 0 : ((lv.order[1] == q) ? 1 : 2);
        const int posr = (lv.order[0] == r) ? 0 : ((lv.order[1] == r) ? 1 : 2);
        a += tune_pass<A, S>(v, cubic, d, (posq < p) ? S : 2 * S, (posr < p) ? S : 2 * S, e);
    }
    acc[LV] = a;
    if constexpr (LV > 0) tune_levels<A, LV - 1>(v, lv, e, acc);
}

// One auto-tune block: sample `sample` (of m, every stride-th tile in
// row-major order) is loaded once and candidates group, group + groups, ...
// are evaluated on it in turn; the per-level sums go to
// err[sample][l][c].  The last of the field's m * groups blocks (ticket) sums
// over the samples and writes each level's argmin to hdr->level (ties to the
// first candidate), then resets the ticket.  v: (A+1)^3 floats of dynamic
// shared memory.
template <int A>
__device__ __forceinline__ void tune_sample(float* v, const CUtensorMap* tmap, const FieldGeo& g,
                                            const float* __restrict__ x, const TuneCands& cands, int sample,
                                            int group, int groups, int stride, int m, double* __restrict__ err,
                                            uint32_t* ticket, hi_header* __restrict__ hdr, uint32_t tma_bytes,
                                            bool use_tma)
{
    using TG = TileGeom<A>;
    constexpr int L = TG::L;
    __shared__ double s_red[L][16];  // up to 512 threads
    __shared__ __align__(8) uint64_t s_mbar;
    __shared__ bool s_last;
    __shared__ double s_tot[L * kMaxCands];

    const int tile = sample * stride;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    int t[3], o[3], e[3];
    tile_coords_rm(g, tile, t);
    for (int d = 0; d < 3; ++d) {
        o[d] = t[d] * A;
        const int rem = (int)(g.n[d] - 1 - o[d]);
        e[d] = (g.n[d] == 1) ? 0 : (rem < A ? rem : A);
    }
    if (use_tma) {  // one TMA box for the sampled tile
        if (tid == 0) {
            mbar_init(&s_mbar, 1);
            fence_mbar_init();
            mbar_arrive_expect_tx(&s_mbar, tma_bytes);
            tma_load_3d(v, tmap, o[2], o[1], o[0], &s_mbar);
        }
        __syncthreads();
        const bool ok = mbar_wait(&s_mbar, 0, kSpinLimit);
        if (!__syncthreads_and(ok)) {
            // the copy may still be in flight: stay until it lands
            if (tid == 0) set_status(&hdr->status, HI_ETIMEOUT);
            drain_wait(&s_mbar, 0);
            __syncthreads();
            return;
        }
    } else {
        const int rows = (e[0] + 1) * (e[1] + 1);
        for (int rr = warp; rr < rows; rr += (blockDim.x >> 5)) {
            const int c0 = rr / (e[1] + 1), c1 = rr - c0 * (e[1] + 1);
            const float* src = x + ((int64_t)(o[0] + c0) * g.n[1] + (o[1] + c1)) * g.n[2] + o[2];
            for (int c2 = lane; c2 <= e[2]; c2 += 32) cp_async4(v + c0 * TG::PY + c1 * TG::PX + c2, src + c2);
        }
        cp_async_wait_all();
        __syncthreads();
    }

    const int ncfg = cands.ncfg;
    for (int c = group; c < ncfg; c += groups) {
        hi_level lv;
        lv.interp = cands.interp[c];
        lv.order[0] = cands.order[c][0];
        lv.order[1] = cands.order[c][1];
        lv.order[2] = cands.order[c][2];
        double acc[L];
        tune_levels<A, L - 1>(v, lv, e, acc);
        // fixed-order reduction: warp butterfly, then warps in index order
#pragma unroll
        for (int l = 0; l < L; ++l) {
            double a = acc[l];
            for (int off = 16; off > 0; off >>= 1) a += __shfl_down_sync(0xffffffffu, a, off);
            if (lane == 0) s_red[l][warp] = a;
        }
        __syncthreads();
        if (tid < L) {
            double a = 0.0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) a += s_red[tid][w];
            err[((size_t)sample * L + tid) * ncfg + c] = a;
        }
        __syncthreads();  // s_red is reused by the next candidate
    }

    // the last block of the field sums the samples and picks each level's candidate
    __threadfence();
    __syncthreads();
    if (tid == 0) s_last = atomicAdd(ticket, 1u) == (uint32_t)(m * groups) - 1;
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int pr = warp; pr < L * ncfg; pr += (blockDim.x >> 5)) {  // one warp per (level, candidate)
        const int l = pr / ncfg, cc = pr - l * ncfg;
        double a = 0.0;
        for (int k = lane; k < m; k += 32) a += __ldcg(err + ((size_t)k * L + l) * ncfg + cc);
        for (int off = 16; off > 0; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
        if (lane == 0) s_tot[pr] = a;
    }
    __syncthreads();
    if (tid < L) {  // smallest sum, ties to the first candidate
        int best = 0;
        for (int cc = 1; cc < ncfg; ++cc)
            if (s_tot[tid * ncfg + cc] < s_tot[tid * ncfg + best]) best = cc;
        hi_level lb;
        lb.interp = cands.interp[best];
        lb.order[0] = cands.order[best][0];
        lb.order[1] = cands.order[best][1];
        lb.order[2] = cands.order[best][2];
        hdr->level[tid] = lb;
    }
    if (tid == 0) *ticket = 0;
}

}  // namespace hi
