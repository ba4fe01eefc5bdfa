// hi_fast.cuh -- level passes for whole interior tiles (extent A in every
// dim, no owned upper face) of the interpolation predictor / quantizer and
// its inverse (cuSZ-Hi, arXiv 2507.11165, Sec. 3.2, Sec. 5.1.1-5.1.2,
// Sec. 5.2.1), in packed two-lane FP32 arithmetic.
//
// Every pass of such a tile has its line counts, stencil cases and
// shared-memory offsets fixed at compile time.  A thread takes two lines of
// the pass at a time whose points have the same stencil case, so that every
// add and subtract of the prediction and of the quantizer is one packed
// f32x2 instruction for two points (products stay scalar, see p_mul).  The
// packed add / sub round each lane on its own (round to nearest even) exactly
// as the scalar operations do, and nothing is contracted into a multiply-add,
// so the results are the ones of the fixed evaluation order the method
// depends on (Eq. 1: the decompressor repeats the compressor's arithmetic bit
// for bit).
//
// Line pairs:
//   * lines along d0 / d1 whose neighbours along d2 are both on the pass
//     (d2 refined earlier in the level, stride 1) -- two adjacent columns,
//     loaded and stored as 8-byte pairs; the columns at d2 = A are paired
//     along the other dim;
//   * all other lines -- line i with line i + ceil(n/2) (adjacent lanes take
//     adjacent lines); rows along d2 are read with 16-byte loads.
// A pass with an odd line count repeats its last line in the second lane
// (same values written twice; its codes are stored once).
//
// Compression stages the codes of the tile's owned points (local coordinates
// below A in every dim) in an A^3 byte box with rows of A bytes; the epilogue
// stores it with vector stores, counts the histogram and, only in tiles where
// a point failed the quantizer, collects the outliers.
#pragma once

#include "hi_passes.cuh"

// Level functions of the fast passes: out of line unless the including
// kernel has the registers to take them inline.
#ifndef HI_FAST_FN
#define HI_FAST_FN __noinline__
#endif

namespace hi {

// ---------------------------------------------------------------------------
// Packed pairs
// ---------------------------------------------------------------------------
// Adds and subtracts are single packed f32x2 instructions (explicit .rn).
// Products are two scalar multiplies: a packed multiply feeding a packed add
// is fused into a packed multiply-add by the assembler even with explicit
// rounding and -fmad=false (measured on sm_103a: the sums came out as
// fmaf's), while the scalar __fmul_rn is never merged into a multiply-add.
// So no product is ever rounded together with the sum that consumes it.
#define HI_F32X2_OP(name, op)                                                        \
    __device__ __forceinline__ float2 name(float2 a, float2 b)                       \
    {                                                                                \
        float2 r;                                                                    \
        asm("{\n\t.reg .b64 pa, pb, pd;\n\t"                                        \
            "mov.b64 pa, {%2, %3};\n\t"                                              \
            "mov.b64 pb, {%4, %5};\n\t" op " pd, pa, pb;\n\t"                       \
            "mov.b64 {%0, %1}, pd;\n\t}"                                             \
            : "=f"(r.x), "=f"(r.y)                                                   \
            : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));                               \
        return r;                                                                    \
    }
HI_F32X2_OP(p_add, "add.rn.f32x2")
HI_F32X2_OP(p_sub, "sub.rn.f32x2")
#undef HI_F32X2_OP
__device__ __forceinline__ float2 p_mul(float2 a, float2 b)
{
    return make_float2(__fmul_rn(a.x, b.x), __fmul_rn(a.y, b.y));
}
__device__ __forceinline__ float2 p_dup(float c) { return make_float2(c, c); }

// A group of threads that runs the passes of one tile together: its size T,
// the calling thread's index in it (its threads are FIRST .. FIRST + T - 1 of
// the CTA) and its barrier: BAR = 0 the whole CTA (__syncthreads), BAR < 0 one
// warp (__syncwarp), BAR > 0 the named barrier BAR over the group's T threads.
template <int N, int FIRST, int BAR>
struct Grp {
    static constexpr int T = N;
    __device__ __forceinline__ static int tid() { return (int)threadIdx.x - FIRST; }
    __device__ __forceinline__ static void sync()
    {
        if constexpr (BAR == 0)
            __syncthreads();
        else if constexpr (BAR < 0)
            __syncwarp();
        else
            asm volatile("bar.sync %0, %1;" ::"n"(BAR), "n"(N) : "memory");
    }
    // barrier with an OR over the group's predicates
    __device__ __forceinline__ static bool sync_or(bool p)
    {
        if constexpr (BAR == 0) {
            return __syncthreads_or(p) != 0;
        } else if constexpr (BAR < 0) {
            return __any_sync(0xffffffffu, p);
        } else {
            uint32_t r;
            asm volatile(
                "{\n\t.reg .pred pi, po;\n\t"
                "setp.ne.u32 pi, %1, 0;\n\t"
                "barrier.red.or.pred po, %2, %3, pi;\n\t"
                "selp.u32 %0, 1, 0, po;\n\t}"
                : "=r"(r)
                : "r"((uint32_t)p), "n"(BAR), "n"(N)
                : "memory");
            return r != 0;
        }
    }
};

// Rounding addend whose low mantissa byte is the code: fl(t + M) = M + rint(t)
// for |t| < 2^22 - 128 (unit spacing in [2^23, 2^24), M even, so ties go to
// even as in rint); its bit pattern is 0x4B400080 + q, whose low byte is
// q + 128 for q in [-127, 127].
constexpr float kCodeMagic = 12583040.0f;  // 1.5 * 2^23 + 128
constexpr uint32_t kCodeBits = 0x4B400000u;  // bits of 1.5 * 2^23; | code = bits of 1.5 * 2^23 + code

struct FastC {
    float2 r;     // 1 / (2 eps) in both lanes
    float2 ebx2;  // 2 eps
    float2 M;     // kCodeMagic
    float2 nM;    // -kCodeMagic
    float eb_f;
};

__device__ __forceinline__ FastC fast_consts(const Hot& h)
{
    FastC c;
    c.r = p_dup(h.r_f);
    c.ebx2 = p_dup(h.ebx2_f);
    c.M = p_dup(kCodeMagic);
    c.nM = p_dup(-kCodeMagic);
    c.eb_f = h.eb_f;
    return c;
}

// Stencil cases of a whole line (Sec. 5.1.2): 0 midpoint (b + u) / 2,
// 1 cubic (-1, 9, 9, -1) / 16, 2 quadratic without f(c-3s) (3, 6, -1) / 8,
// 3 quadratic without f(c+3s) (-1, 6, 3) / 8.  Point k of NDM on a line of
// extent A has f(c-3s) iff k >= 1 and f(c+3s) iff k <= NDM - 2.
__host__ __device__ constexpr int fcase(bool cubic, int ndm, int k)
{
    return (!cubic || ndm == 1) ? 0 : (k == 0 ? 2 : (k == ndm - 1 ? 3 : 1));
}

template <int C>
__device__ __forceinline__ float2 pred2(float2 a, float2 b, float2 u, float2 v)
{
    if constexpr (C == 0) {
        return p_mul(p_add(b, u), p_dup(0.5f));
    } else if constexpr (C == 1) {
        return p_mul(p_sub(p_mul(p_dup(9.0f), p_add(b, u)), p_add(a, v)), p_dup(0.0625f));
    } else if constexpr (C == 2) {
        return p_mul(p_sub(p_add(p_mul(p_dup(3.0f), b), p_mul(p_dup(6.0f), u)), v), p_dup(0.125f));
    } else {
        return p_mul(p_sub(p_add(p_mul(p_dup(6.0f), b), p_mul(p_dup(3.0f), u)), a), p_dup(0.125f));
    }
}

// Linear quantization of two points (Sec. 5.2.1), the same operations as
// quantize(): t = (x - p) r, q = rint(t), x' = p + q 2eps; an outlier when
// !(|t| < 127.5) or !(|x - x'| < eb_f).  Returns the reconstructed pair;
// ca / cb get the code in their low byte (0 for an outlier); bad is set when
// either point is an outlier.
__device__ __forceinline__ float2 quant2(float2 x, float2 p, const FastC& c, uint32_t& ca, uint32_t& cb, bool& bad)
{
    const float2 t = p_mul(p_sub(x, p), c.r);
    const float2 m = p_add(t, c.M);
    const float2 qf = p_add(m, c.nM);
    const float2 xr = p_add(p, p_mul(qf, c.ebx2));
    const float2 d = p_sub(x, xr);
    const bool oka = (fabsf(t.x) < kQmax) && (fabsf(d.x) < c.eb_f);
    const bool okb = (fabsf(t.y) < kQmax) && (fabsf(d.y) < c.eb_f);
    ca = oka ? __float_as_uint(m.x) : 0u;
    cb = okb ? __float_as_uint(m.y) : 0u;
    bad = bad || !(oka && okb);
    return make_float2(oka ? xr.x : x.x, okb ? xr.y : x.y);
}

// Reconstruction of two points from their codes, given as 0x4B4000cc (the
// code in the low byte): (1.5 * 2^23 + code) - (1.5 * 2^23 + 128) is
// code - 128 exactly, then x' = p + q 2eps as in dequantize().
__device__ __forceinline__ float2 dequant2(uint32_t ba, uint32_t bb, float2 p, const FastC& c)
{
    const float2 qf = p_add(make_float2(__uint_as_float(ba), __uint_as_float(bb)), c.nM);
    return p_add(p, p_mul(qf, c.ebx2));
}

// ---------------------------------------------------------------------------
// Layout of the staged tile seen by the fast passes
// ---------------------------------------------------------------------------
template <int A, bool COMP>
struct FLay {
    using Lw = Lay<A>;
    // float pitches of dims 0, 1, 2 in the tile buffer
    static constexpr int V0 = Lw::PY, V1 = Lw::PX;
    // code pitches: compression's owned A^3 box, decompression's staged tile
    static constexpr int K0 = COMP ? A * A : Lw::CYD;
    static constexpr int K1 = COMP ? A : Lw::CXD;
    __host__ __device__ static constexpr int v(int d) { return d == 0 ? V0 : (d == 1 ? V1 : 1); }
    __host__ __device__ static constexpr int k(int d) { return d == 0 ? K0 : (d == 1 ? K1 : 1); }
};

__device__ __forceinline__ float2 lds2(const float* p) { return *reinterpret_cast<const float2*>(p); }
__device__ __forceinline__ void sts2(float* p, float2 a) { *reinterpret_cast<float2*>(p) = a; }

// One pair of lines along D (not d2), starting at float offsets va, vb and
// code offsets ka, kb.  VEC: the two lines are adjacent along d2 (vb = va + 1,
// va even).  COMP: ownA / ownB say whether the lines' codes are stored.
template <int A, int S, int D, bool CUBIC, bool COMP, bool VEC>
__device__ __forceinline__ void col_pair(float* __restrict__ v, uint8_t* __restrict__ cs, const FastC& c, int va,
                                         int vb, int ka, int kb, bool ownA, bool ownB, bool& bad)
{
    using FL = FLay<A, COMP>;
    constexpr int NDM = A / (2 * S);
    constexpr int VD = FL::v(D) * S, KD = FL::k(D) * S;
    float2 f[NDM + 1];
#pragma unroll
    for (int m = 0; m <= NDM; ++m) {
        if constexpr (VEC)
            f[m] = lds2(v + va + 2 * m * VD);
        else
            f[m] = make_float2(v[va + 2 * m * VD], v[vb + 2 * m * VD]);
    }
#pragma unroll
    for (int k = 0; k < NDM; ++k) {
        const float2 a = f[k >= 1 ? k - 1 : 0], b = f[k], u = f[k + 1], w = f[k + 2 <= NDM ? k + 2 : NDM];
        float2 p;
        switch (fcase(CUBIC, NDM, k)) {
        case 0: p = pred2<0>(a, b, u, w); break;
        case 1: p = pred2<1>(a, b, u, w); break;
        case 2: p = pred2<2>(a, b, u, w); break;
        default: p = pred2<3>(a, b, u, w); break;
        }
        const int o = (2 * k + 1) * VD, ok = (2 * k + 1) * KD;
        if constexpr (COMP) {
            const float2 x = VEC ? lds2(v + va + o) : make_float2(v[va + o], v[vb + o]);
            uint32_t ca, cb;
            const float2 r = quant2(x, p, c, ca, cb, bad);
            if constexpr (VEC) {
                sts2(v + va + o, r);
                if (ownA) *reinterpret_cast<uint16_t*>(cs + ka + ok) = (uint16_t)__byte_perm(ca, cb, 0x40);
            } else {
                v[va + o] = r.x;
                v[vb + o] = r.y;
                if (ownA) cs[ka + ok] = (uint8_t)ca;
                if (ownB) cs[kb + ok] = (uint8_t)cb;
            }
        } else {
            uint32_t ba, bb;
            if constexpr (VEC) {
                const uint32_t w2 = *reinterpret_cast<const uint16_t*>(cs + ka + ok);
                ba = __byte_perm(w2, kCodeBits, 0x7650);
                bb = __byte_perm(w2, kCodeBits, 0x7651);
            } else {
                ba = kCodeBits | cs[ka + ok];
                bb = kCodeBits | cs[kb + ok];
            }
            const float2 r = dequant2(ba, bb, p, c);
            if constexpr (VEC) {
                sts2(v + va + o, r);
            } else {
                v[va + o] = r.x;
                v[vb + o] = r.y;
            }
        }
    }
}

// One pair of rows (lines along d2) at float offsets va, vb, code offsets
// ka, kb.  Rows at strides 1 and 2 are read and (stride 1) written with
// 16-byte accesses.
template <int A, int S, bool CUBIC, bool COMP>
__device__ __forceinline__ void row_pair(float* __restrict__ v, uint8_t* __restrict__ cs, const FastC& c, int va,
                                         int vb, int ka, int kb, bool ownA, bool ownB, bool& bad)
{
    constexpr int NDM = A / (2 * S);
    constexpr bool WIDE = (S <= 2);  // read the whole row
    float ra[A + 1], rb[A + 1];
    if constexpr (WIDE) {
#pragma unroll
        for (int j = 0; j < A / 4; ++j) {
            const float4 qa = reinterpret_cast<const float4*>(v + va)[j];
            const float4 qb = reinterpret_cast<const float4*>(v + vb)[j];
            ra[4 * j] = qa.x, ra[4 * j + 1] = qa.y, ra[4 * j + 2] = qa.z, ra[4 * j + 3] = qa.w;
            rb[4 * j] = qb.x, rb[4 * j + 1] = qb.y, rb[4 * j + 2] = qb.z, rb[4 * j + 3] = qb.w;
        }
        ra[A] = v[va + A];
        rb[A] = v[vb + A];
    } else {
#pragma unroll
        for (int j = 0; j <= A; j += S) {
            ra[j] = v[va + j];
            rb[j] = v[vb + j];
        }
    }
    uint32_t wa[(A + 3) / 4], wb[(A + 3) / 4];  // decompression: codes 0 .. A-1 of the rows, 4 per word
    if constexpr (!COMP) {
        if constexpr (A == 16) {
            const uint4 qa = *reinterpret_cast<const uint4*>(cs + ka);
            const uint4 qb = *reinterpret_cast<const uint4*>(cs + kb);
            wa[0] = qa.x, wa[1] = qa.y, wa[2] = qa.z, wa[3] = qa.w;
            wb[0] = qb.x, wb[1] = qb.y, wb[2] = qb.z, wb[3] = qb.w;
        } else {
            static_assert(A == 8, "row codes");
            const uint2 qa = *reinterpret_cast<const uint2*>(cs + ka);
            const uint2 qb = *reinterpret_cast<const uint2*>(cs + kb);
            wa[0] = qa.x, wa[1] = qa.y;
            wb[0] = qb.x, wb[1] = qb.y;
        }
    }
#pragma unroll
    for (int k = 0; k < NDM; ++k) {
        const int cc = (2 * k + 1) * S;
        const float2 a = make_float2(ra[k >= 1 ? cc - 3 * S : 0], rb[k >= 1 ? cc - 3 * S : 0]);
        const float2 b = make_float2(ra[cc - S], rb[cc - S]);
        const float2 u = make_float2(ra[cc + S], rb[cc + S]);
        const int iw = (cc + 3 * S <= A) ? cc + 3 * S : A;
        const float2 w = make_float2(ra[iw], rb[iw]);
        float2 p;
        switch (fcase(CUBIC, NDM, k)) {
        case 0: p = pred2<0>(a, b, u, w); break;
        case 1: p = pred2<1>(a, b, u, w); break;
        case 2: p = pred2<2>(a, b, u, w); break;
        default: p = pred2<3>(a, b, u, w); break;
        }
        float2 r;
        if constexpr (COMP) {
            uint32_t ca, cb;
            r = quant2(make_float2(ra[cc], rb[cc]), p, c, ca, cb, bad);
            if (ownA) cs[ka + cc] = (uint8_t)ca;
            if (ownB) cs[kb + cc] = (uint8_t)cb;
        } else {
            const uint32_t sel = 0x7650u | (uint32_t)(cc & 3);
            r = dequant2(__byte_perm(wa[cc >> 2], kCodeBits, sel), __byte_perm(wb[cc >> 2], kCodeBits, sel), p, c);
        }
        ra[cc] = r.x;
        rb[cc] = r.y;
    }
    if constexpr (S == 1) {
#pragma unroll
        for (int j = 0; j < A / 4; ++j) {
            reinterpret_cast<float4*>(v + va)[j] = make_float4(ra[4 * j], ra[4 * j + 1], ra[4 * j + 2], ra[4 * j + 3]);
            reinterpret_cast<float4*>(v + vb)[j] = make_float4(rb[4 * j], rb[4 * j + 1], rb[4 * j + 2], rb[4 * j + 3]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < NDM; ++k) {
            const int cc = (2 * k + 1) * S;
            v[va + cc] = ra[cc];
            v[vb + cc] = rb[cc];
        }
    }
}

// Step of dim d in pass P of a level with sequence (D0, D1, D2).
template <int D0, int D1, int D2, int P, int S>
__host__ __device__ constexpr int fstep(int d)
{
    return ((d == D0 ? 0 : (d == D1 ? 1 : 2)) < P) ? S : 2 * S;
}

// One pass (dim D, pass P of the level's sequence) over a whole tile by T threads.
template <int A, int S, int P, int D0, int D1, int D2, bool CUBIC, bool COMP, class G>
__device__ __forceinline__ void fpass(float* __restrict__ v, uint8_t* __restrict__ cs, const FastC& c, bool& bad)
{
    using FL = FLay<A, COMP>;
    constexpr int D = (P == 0) ? D0 : (P == 1 ? D1 : D2);
    constexpr int Q = (D == 0) ? 1 : 0, R = (D == 2) ? 1 : 2;  // the other dims, Q < R
    constexpr int STQ = fstep<D0, D1, D2, P, S>(Q), STR = fstep<D0, D1, D2, P, S>(R);
    constexpr int NQ = A / STQ + 1, NR = A / STR + 1, NL = NQ * NR;
    constexpr int VQ = FL::v(Q) * STQ, VR = FL::v(R) * STR;
    constexpr int KQ = FL::k(Q) * STQ, KR = FL::k(R) * STR;
    constexpr bool ADJ = (D != 2) && (STR == 1);
    if constexpr (ADJ) {
        // columns (jq, 2i) and (jq, 2i + 1) for 2i + 1 < A; then the columns at
        // d2 = A paired along Q
        constexpr int NPR = A / 2;
        constexpr int NV = NQ * NPR;
        constexpr int NS = (NQ + 1) / 2;
        constexpr int NI = NV + NS;
#pragma unroll
        for (int r0 = 0; r0 < NI; r0 += G::T) {
            const int it = r0 + G::tid();
            if (it < NV) {
                const int jq = it / NPR, i2 = 2 * (it - jq * NPR);
                const int va = jq * VQ + i2, ka = jq * KQ + i2;
                const bool own = jq * STQ < A;
                col_pair<A, S, D, CUBIC, COMP, true>(v, cs, c, va, va + 1, ka, ka + 1, own, own, bad);
            } else if (it < NI) {
                const int j = it - NV;
                const int qa = 2 * j, qb = (2 * j + 1 < NQ) ? 2 * j + 1 : 2 * j;
                col_pair<A, S, D, CUBIC, COMP, false>(v, cs, c, qa * VQ + A, qb * VQ + A, qa * KQ + A, qb * KQ + A,
                                                      false, false, bad);
            }
        }
    } else {
        constexpr int NH = (NL + 1) / 2;  // pairs: line i with line i + NH
#pragma unroll
        for (int r0 = 0; r0 < NH; r0 += G::T) {
            const int it = r0 + G::tid();
            if (it < NH) {
                const int la = it, lb = (it + NH < NL) ? it + NH : it;
                const int qa = la / NR, qb = lb / NR;
                const int ja = la - qa * NR, jb = lb - qb * NR;
                const int va = qa * VQ + ja * VR, vb = qb * VQ + jb * VR;
                const int ka = qa * KQ + ja * KR, kb = qb * KQ + jb * KR;
                const bool ownA = qa * STQ < A && ja * STR < A;
                const bool ownB = lb != la && qb * STQ < A && jb * STR < A;
                if constexpr (D == 2)
                    row_pair<A, S, CUBIC, COMP>(v, cs, c, va, vb, ka, kb, ownA, ownB, bad);
                else
                    col_pair<A, S, D, CUBIC, COMP, false>(v, cs, c, va, vb, ka, kb, ownA, ownB, bad);
            }
        }
    }
}

// The multi-dimensional scheme (Sec. 5.1.2) on a whole tile with the fast
// path's code layout: the points whose odd dims are the set M (see
// md_set_full); codes of owned points only.  Scalar arithmetic: the points of
// a phase do not share a stencil case.
template <int A, int S, int M, bool CUBIC, bool COMP, class G>
__device__ __forceinline__ void md_set_owned(float* v, uint8_t* cs, const Hot h, bool& bad)
{
    using Lw = Lay<A>;
    using FL = FLay<A, COMP>;
    constexpr int NO = A / (2 * S), NE = A / (2 * S) + 1;
    constexpr int N0 = (M & 1) ? NO : NE, N1 = (M & 2) ? NO : NE, N2 = (M & 4) ? NO : NE;
    constexpr int TOTAL = N0 * N1 * N2;
    for (int i = G::tid(); i < TOTAL; i += G::T) {
        const int j2 = i % N2, r = i / N2;
        const int j1 = r % N1, j0 = r / N1;
        const int c0 = (M & 1) ? (2 * j0 + 1) * S : 2 * j0 * S;
        const int c1 = (M & 2) ? (2 * j1 + 1) * S : 2 * j1 * S;
        const int c2 = (M & 4) ? (2 * j2 + 1) * S : 2 * j2 * S;
        const int vi = c0 * Lw::PY + c1 * Lw::PX + c2;
        const int jd[3] = {j0, j1, j2};
        float p[3];
        int o[3];
        int best = -1;
#pragma unroll
        for (int d = 0; d < 3; ++d) {
            p[d] = 0.0f;
            o[d] = -1;
            if (!((M >> d) & 1)) continue;
            const int st = (d == 0 ? Lw::PY : (d == 1 ? Lw::PX : 1)) * S;
            const bool l3 = CUBIC && jd[d] >= 1, r3 = CUBIC && jd[d] <= NO - 2;
            const float b = v[vi - st], u = v[vi + st];
            const float a = l3 ? v[vi - 3 * st] : 0.0f;
            const float w = r3 ? v[vi + 3 * st] : 0.0f;
            p[d] = predict(CUBIC, l3, true, r3, a, b, u, w);
            o[d] = !CUBIC ? 1 : ((l3 && r3) ? 3 : ((l3 || r3) ? 2 : 1));
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
        const int ci = c0 * FL::K0 + c1 * FL::K1 + c2;
        if constexpr (COMP) {
            float xr;
            const int code = quantize(v[vi], pr, h.eb_f, h.ebx2_f, h.r_f, xr);
            v[vi] = xr;
            bad = bad || code == 0;
            if (c0 < A && c1 < A && c2 < A) cs[ci] = (uint8_t)code;
        } else {
            v[vi] = dequantize(cs[ci], pr, h.ebx2_f);
        }
    }
}

template <int A, int S, bool CUBIC, bool COMP, class G>
__device__ HI_FAST_FN bool md_full_owned(float* v, uint8_t* cs, const Hot h)
{
    bool bad = false;
    md_set_owned<A, S, 1, CUBIC, COMP, G>(v, cs, h, bad);  // one odd dim
    md_set_owned<A, S, 2, CUBIC, COMP, G>(v, cs, h, bad);
    md_set_owned<A, S, 4, CUBIC, COMP, G>(v, cs, h, bad);
    G::sync();
    md_set_owned<A, S, 3, CUBIC, COMP, G>(v, cs, h, bad);  // two
    md_set_owned<A, S, 5, CUBIC, COMP, G>(v, cs, h, bad);
    md_set_owned<A, S, 6, CUBIC, COMP, G>(v, cs, h, bad);
    G::sync();
    md_set_owned<A, S, 7, CUBIC, COMP, G>(v, cs, h, bad);  // three
    return bad;
}

// One level: three passes with a barrier of the group after the first two
// (the caller places the one after the third).  Returns whether a point of
// this thread was an outlier (compression).
template <int A, int S, int D0, int D1, int D2, bool CUBIC, bool COMP, class G>
__device__ HI_FAST_FN bool flevel(float* v, uint8_t* cs, const FastC c)
{
    bool bad = false;
    fpass<A, S, 0, D0, D1, D2, CUBIC, COMP, G>(v, cs, c, bad);
    G::sync();
    fpass<A, S, 1, D0, D1, D2, CUBIC, COMP, G>(v, cs, c, bad);
    G::sync();
    fpass<A, S, 2, D0, D1, D2, CUBIC, COMP, G>(v, cs, c, bad);
    return bad;
}

// sel = 2 * perm + cubic (perm: 0 (0,1,2) 1 (0,2,1) 2 (1,0,2) 3 (1,2,0) 4 (2,0,1) 5 (2,1,0));
// 12 / 13: the multi-dimensional scheme with linear / cubic splines
template <int A, int S, bool COMP, class G>
__device__ __forceinline__ bool flevel_dispatch(int sel, float* v, uint8_t* cs, const FastC& c, const Hot h)
{
    switch (sel) {
    case 0: return flevel<A, S, 0, 1, 2, false, COMP, G>(v, cs, c);
    case 1: return flevel<A, S, 0, 1, 2, true, COMP, G>(v, cs, c);
    case 2: return flevel<A, S, 0, 2, 1, false, COMP, G>(v, cs, c);
    case 3: return flevel<A, S, 0, 2, 1, true, COMP, G>(v, cs, c);
    case 4: return flevel<A, S, 1, 0, 2, false, COMP, G>(v, cs, c);
    case 5: return flevel<A, S, 1, 0, 2, true, COMP, G>(v, cs, c);
    case 6: return flevel<A, S, 1, 2, 0, false, COMP, G>(v, cs, c);
    case 7: return flevel<A, S, 1, 2, 0, true, COMP, G>(v, cs, c);
    case 8: return flevel<A, S, 2, 0, 1, false, COMP, G>(v, cs, c);
    case 9: return flevel<A, S, 2, 0, 1, true, COMP, G>(v, cs, c);
    case 10: return flevel<A, S, 2, 1, 0, false, COMP, G>(v, cs, c);
    case 11: return flevel<A, S, 2, 1, 0, true, COMP, G>(v, cs, c);
    case 12: return md_full_owned<A, S, false, COMP, G>(v, cs, h);
    default: return md_full_owned<A, S, true, COMP, G>(v, cs, h);
    }
}

// Levels HI .. LO of a whole tile, coarsest first, with a group barrier
// between levels and none after the last pass.  Returns this thread's
// outlier flag.
template <int A, int HI, int LO, bool COMP, class G>
__device__ __forceinline__ bool flevels(const int* s_sel, float* v, uint8_t* cs, const FastC& c, const Hot h)
{
    bool bad = flevel_dispatch<A, (1 << HI), COMP, G>(s_sel[HI], v, cs, c, h);
    if constexpr (HI > LO) {
        G::sync();
        bad = flevels<A, HI - 1, LO, COMP, G>(s_sel, v, cs, c, h) || bad;
    }
    return bad;
}

// ---------------------------------------------------------------------------
// Coarse levels by a small group: one line per thread, scalar arithmetic.  A
// coarse pass has a few dozen lines of one to four points; single lines keep
// more of the group's lanes busy than line pairs would.
// ---------------------------------------------------------------------------
template <int A, int S, int P, int D0, int D1, int D2, bool CUBIC, bool COMP, class G>
__device__ __forceinline__ void spass(float* __restrict__ v, uint8_t* __restrict__ cs, const Hot h, bool& bad)
{
    using FL = FLay<A, COMP>;
    constexpr int D = (P == 0) ? D0 : (P == 1 ? D1 : D2);
    constexpr int Q = (D == 0) ? 1 : 0, R = (D == 2) ? 1 : 2;
    constexpr int STQ = fstep<D0, D1, D2, P, S>(Q), STR = fstep<D0, D1, D2, P, S>(R);
    constexpr int NQ = A / STQ + 1, NR = A / STR + 1, NL = NQ * NR;
    constexpr int NDM = A / (2 * S);
    constexpr int VD = FL::v(D) * S, KD = FL::k(D) * S;
    for (int l = G::tid(); l < NL; l += G::T) {
        const int jq = l / NR, jr = l - (l / NR) * NR;
        const int cq = jq * STQ, cr = jr * STR;
        const int vb = cq * FL::v(Q) + cr * FL::v(R), kb = cq * FL::k(Q) + cr * FL::k(R);
        const bool own = cq < A && cr < A;
        float f[NDM + 1];
#pragma unroll
        for (int m = 0; m <= NDM; ++m) f[m] = v[vb + 2 * m * VD];
#pragma unroll
        for (int k = 0; k < NDM; ++k) {
            const float pr = predict(CUBIC, k >= 1, true, k <= NDM - 2, f[k >= 1 ? k - 1 : 0], f[k], f[k + 1],
                                     f[k + 2 <= NDM ? k + 2 : NDM]);
            const int vi = vb + (2 * k + 1) * VD;
            if constexpr (COMP) {
                float xr;
                const int code = quantize(v[vi], pr, h.eb_f, h.ebx2_f, h.r_f, xr);
                v[vi] = xr;
                bad = bad || code == 0;
                if (own) cs[kb + (2 * k + 1) * KD] = (uint8_t)code;
            } else {
                v[vi] = dequantize(cs[kb + (2 * k + 1) * KD], pr, h.ebx2_f);
            }
        }
    }
}

template <int A, int S, int D0, int D1, int D2, bool CUBIC, bool COMP, class G>
__device__ HI_FAST_FN bool slevel(float* v, uint8_t* cs, const Hot h)
{
    bool bad = false;
    spass<A, S, 0, D0, D1, D2, CUBIC, COMP, G>(v, cs, h, bad);
    G::sync();
    spass<A, S, 1, D0, D1, D2, CUBIC, COMP, G>(v, cs, h, bad);
    G::sync();
    spass<A, S, 2, D0, D1, D2, CUBIC, COMP, G>(v, cs, h, bad);
    return bad;
}

template <int A, int S, bool COMP, class G>
__device__ __forceinline__ bool slevel_dispatch(int sel, float* v, uint8_t* cs, const Hot h)
{
    switch (sel) {
    case 0: return slevel<A, S, 0, 1, 2, false, COMP, G>(v, cs, h);
    case 1: return slevel<A, S, 0, 1, 2, true, COMP, G>(v, cs, h);
    case 2: return slevel<A, S, 0, 2, 1, false, COMP, G>(v, cs, h);
    case 3: return slevel<A, S, 0, 2, 1, true, COMP, G>(v, cs, h);
    case 4: return slevel<A, S, 1, 0, 2, false, COMP, G>(v, cs, h);
    case 5: return slevel<A, S, 1, 0, 2, true, COMP, G>(v, cs, h);
    case 6: return slevel<A, S, 1, 2, 0, false, COMP, G>(v, cs, h);
    case 7: return slevel<A, S, 1, 2, 0, true, COMP, G>(v, cs, h);
    case 8: return slevel<A, S, 2, 0, 1, false, COMP, G>(v, cs, h);
    case 9: return slevel<A, S, 2, 0, 1, true, COMP, G>(v, cs, h);
    case 10: return slevel<A, S, 2, 1, 0, false, COMP, G>(v, cs, h);
    case 11: return slevel<A, S, 2, 1, 0, true, COMP, G>(v, cs, h);
    case 12: return md_full_owned<A, S, false, COMP, G>(v, cs, h);
    default: return md_full_owned<A, S, true, COMP, G>(v, cs, h);
    }
}

// Levels HI .. LO (coarse strides) by a small group, coarsest first.
template <int A, int HI, int LO, bool COMP, class G>
__device__ __forceinline__ bool slevels(const int* s_sel, float* v, uint8_t* cs, const Hot h)
{
    bool bad = slevel_dispatch<A, (1 << HI), COMP, G>(s_sel[HI], v, cs, h);
    if constexpr (HI > LO) {
        G::sync();
        bad = slevels<A, HI - 1, LO, COMP, G>(s_sel, v, cs, h) || bad;
    }
    return bad;
}

// Fast tiles: whole in every dim and not the last block along any dim (so
// the owned points are exactly the A^3 box below the upper faces).
template <int A>
__device__ __forceinline__ bool fast_tile(bool full_ok, const TileInfo& ti)
{
    return HasFull<A>::value && full_ok && ti.e[0] == A && ti.e[1] == A && ti.e[2] == A && ti.own[0] == A - 1 &&
           ti.own[1] == A - 1 && ti.own[2] == A - 1;
}

// ---------------------------------------------------------------------------
// Compression epilogue of a fast tile
// ---------------------------------------------------------------------------
// Histogram: codes 126..129 (the bulk at practical bounds) in the four bytes
// of one register per thread, folded into the CTA histogram every
// kFastFlush tiles (a thread counts at most 2 A codes of a tile); other codes
// by shared-memory atomics.
constexpr uint32_t kFastHotLo = 126;
constexpr int kFastFlush = 4;

__device__ __forceinline__ void fast_hist4(uint32_t w, uint32_t& hacc, uint32_t* s_hist)
{
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t code = __byte_perm(w, 0u, 0x4440u | (uint32_t)b);
        const uint32_t sh = code * 8u - 8u * kFastHotLo;
        hacc += __funnelshift_lc(0u, 1u, sh);  // 1 << sh; 0 for sh >= 32 (codes outside 126..129)
        // other codes: a predicated shared-memory reduction, no branch
        asm volatile(
            "{\n\t.reg .pred pc;\n\t"
            "setp.ge.u32 pc, %0, 32;\n\t"
            "@pc red.shared.add.u32 [%1], 1;\n\t}" ::"r"(sh),
            "r"(smem_addr(s_hist + code))
            : "memory");
    }
}

// Fold the register counters into the CTA histogram (whole warps).
__device__ __forceinline__ void fast_hist_flush(uint32_t& hacc, uint32_t* s_hist)
{
#pragma unroll
    for (int b = 0; b < 4; ++b) {
        const uint32_t n = __reduce_add_sync(0xffffffffu, (hacc >> (8 * b)) & 0xffu);
        if ((threadIdx.x & 31) == 0 && n) atomicAdd(&s_hist[kFastHotLo + b], n);
    }
    hacc = 0;
}

// Owned codes (A^3 box, rows of A bytes) to the field's code array, and
// their histogram.  vec_ok: rows may be stored as A-byte vectors.
template <int A, class G>
__device__ __forceinline__ void fast_codes_out(const FieldGeo& g, const TileInfo& ti, const uint8_t* cs,
                                               uint8_t* __restrict__ codes, bool vec_ok, bool hist_on,
                                               uint32_t& hacc, uint32_t* s_hist)
{
    constexpr int NROW = A * A;
#pragma unroll
    for (int r0 = 0; r0 < NROW; r0 += G::T) {
        const int r = r0 + G::tid();
        if (r < NROW) {
            const int c0 = r / A, c1 = r - (r / A) * A;
            uint8_t* dst = codes + ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2];
            uint32_t w[A / 4];
            if constexpr (A == 16) {
                const uint4 q = *reinterpret_cast<const uint4*>(cs + r * A);
                w[0] = q.x, w[1] = q.y, w[2] = q.z, w[3] = q.w;
                if (vec_ok) *reinterpret_cast<uint4*>(dst) = q;
            } else {
                const uint2 q = *reinterpret_cast<const uint2*>(cs + r * A);
                w[0] = q.x, w[1] = q.y;
                if (vec_ok) *reinterpret_cast<uint2*>(dst) = q;
            }
            if (!vec_ok) {
                if ((reinterpret_cast<uintptr_t>(dst) & 3u) == 0) {
#pragma unroll
                    for (int j = 0; j < A / 4; ++j) reinterpret_cast<uint32_t*>(dst)[j] = w[j];
                } else {
#pragma unroll
                    for (int j = 0; j < A; ++j) dst[j] = (uint8_t)(w[j >> 2] >> (8 * (j & 3)));
                }
            }
            if (hist_on) {
#pragma unroll
                for (int j = 0; j < A / 4; ++j) fast_hist4(w[j], hacc, s_hist);
            }
        }
    }
}

// Outliers of a fast tile (code 0 in the owned box; values from the field,
// since an outlier's reconstruction is its own value): a row per lane, the
// warp reserves its slots with one atomic.
template <int A, class G>
__device__ __noinline__ void fast_outliers(const FieldGeo& g, const TileInfo& ti, const uint8_t* cs,
                                           const float* __restrict__ x, hi_header* hdr, uint32_t* out_idx,
                                           float* out_val, uint64_t out_cap)
{
    constexpr int NROW = A * A, NW = A / 4;
    const int lane = threadIdx.x & 31;
    for (int r0 = 0; r0 < NROW; r0 += G::T) {
        const int r = r0 + G::tid();
        const bool act = r < NROW;
        uint32_t zm[NW];
        int cnt = 0;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            const uint32_t w = act ? reinterpret_cast<const uint32_t*>(cs + r * A)[j] : 0x01010101u;
            zm[j] = ~(((w & 0x7f7f7f7fu) + 0x7f7f7f7fu) | w) & 0x80808080u;  // 0x80 in each zero byte
            cnt += __popc(zm[j]);
        }
        if (!__any_sync(0xffffffffu, cnt != 0)) continue;
        int incl = cnt;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, off);
            if (lane >= off) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        unsigned long long base = 0;
        if (lane == 31)
            base = atomicAdd(reinterpret_cast<unsigned long long*>(&hdr->n_outliers), (unsigned long long)total);
        base = __shfl_sync(0xffffffffu, base, 31);
        unsigned long long pos = base + (unsigned long long)(incl - cnt);
        const int c0 = r / A, c1 = r - (r / A) * A;
        const int64_t row = ((int64_t)(ti.o[0] + c0) * g.n[1] + (ti.o[1] + c1)) * g.n[2] + ti.o[2];
        bool over = false;
#pragma unroll
        for (int j = 0; j < NW; ++j) {
            uint32_t m = zm[j];
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                const int64_t gi = row + 4 * j + (bit >> 3);
                if (pos < out_cap) {
                    out_idx[pos] = (uint32_t)gi;
                    out_val[pos] = x[gi];
                } else {
                    over = true;
                }
                ++pos;
            }
        }
        if (over) set_status(&hdr->status, HI_ECAPACITY);
    }
}

}  // namespace hi
