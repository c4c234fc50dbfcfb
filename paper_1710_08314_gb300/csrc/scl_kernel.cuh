// scl_kernel.cuh -- the batched SCL decoding kernel (sm_103a).
//
// One warp decodes 32/L frames at once: lane = frame-in-warp * L + path slot.
// Every lane runs the same node schedule (the pre-order traversal of
// Algorithm 1 with pruned nodes collapsed), so control flow is uniform.
//
// Memory of a warp (Layout):
//  - LLR layer d (d >= 1) holds, for every lane, the 2^(n-d) LLRs of the
//    current depth-d node: row r, column lane, so the 32 lanes of a row are
//    one 128-byte line.  Reads go to the column of the slot the path's layer
//    was written by (lazy path copy by index indirection: a new path inherits
//    its parent's per-layer slot table and writes only its own column).
//  - layer 0 holds the channel LLRs of the warp's frames, column = frame.
//  - BL_d / BR_d hold, bit-packed, the partial sums (Sec. II-B h) of the last
//    completed left / right child at depth d; BL_d is indexed like the LLR
//    layers, BR_d is always the lane's own column.
//  - fixed point packs 2 (int16) or 4 (int8) LLRs per 32-bit word and runs f
//    and g with SIMD-in-word intrinsics.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace pscl {

#define PSCL_FULL 0xFFFFFFFFu

// ---------------------------------------------------------------------------
// Number formats.  Words hold EPW elements of BITS bits; V is the scalar type
// handlers work in.  f and g follow Sec. II-B:
//   f(a, b) = sign(a b) min(|a|, |b|)      g(a, b, s) = (1 - 2s) a + b
// with the sign of f taken from the sign bits and g computed as (s?-a:a)+b.
struct QF32 {
    static constexpr int EPW = 1, BITS = 32, FIXED = 0, VBITS = 0;
    typedef float V;
    __device__ static __forceinline__ uint32_t F(uint32_t a, uint32_t b)
    {
        uint32_t m = __float_as_uint(fminf(fabsf(__uint_as_float(a)), fabsf(__uint_as_float(b))));
        return m | ((a ^ b) & 0x80000000u);
    }
    // s: bit 0 = partial sum of the element
    __device__ static __forceinline__ uint32_t G(uint32_t a, uint32_t b, uint32_t s)
    {
        return __float_as_uint(__fadd_rn(__uint_as_float(a ^ (s << 31)), __uint_as_float(b)));
    }
    __device__ static __forceinline__ V elem(uint32_t w, int) { return __uint_as_float(w); }
    __device__ static __forceinline__ V absv(V v) { return fabsf(v); }
    __device__ static __forceinline__ V add(V a, V b) { return __fadd_rn(a, b); }
    __device__ static __forceinline__ uint32_t key(V v) { return __float_as_uint(v); }
    __device__ static __forceinline__ V from_key(uint32_t k) { return __uint_as_float(k); }
    __device__ static __forceinline__ V zero() { return 0.0f; }
    __device__ static __forceinline__ V big() { return __uint_as_float(0x7F800000u); }
    __device__ static __forceinline__ uint32_t quant(float x) { return __float_as_uint(x); }
    __device__ static __forceinline__ float to_float(V v) { return v; }
    __device__ static __forceinline__ V sub(V a, V) { return a; }
    __device__ static __forceinline__ V f1(V a, V b) { return __uint_as_float(F(__float_as_uint(a), __float_as_uint(b))); }
    __device__ static __forceinline__ V g1(V a, V b, uint32_t s) { return __fadd_rn(s ? -a : a, b); }
};

struct QI16 {
    static constexpr int EPW = 2, BITS = 16, FIXED = 1, Q = 32767, FRAC = 5, VBITS = 15;
    typedef int V;
    __device__ static __forceinline__ uint32_t F(uint32_t a, uint32_t b)
    {
        uint32_t m = __vminu2(__vabsss2(a), __vabsss2(b));
        uint32_t mask = (((a ^ b) & 0x80008000u) >> 15) * 0xFFFFu;
        return (m & ~mask) | (__vneg2(m) & mask);
    }
    // s: bits 0..1 = partial sums of the two elements
    __device__ static __forceinline__ uint32_t G(uint32_t a, uint32_t b, uint32_t s)
    {
        uint32_t mask = ((s & 1u) * 0xFFFFu) | (((s >> 1) & 1u) * 0xFFFF0000u);
        uint32_t na = (a & ~mask) | (__vneg2(a) & mask);
        return __vmaxs2(__vaddss2(na, b), 0x80018001u);  // saturate to [-Q, Q]
    }
    __device__ static __forceinline__ V elem(uint32_t w, int k) { return (int)(int16_t)(w >> (16 * k)); }
    __device__ static __forceinline__ V absv(V v) { return v < 0 ? -v : v; }
    __device__ static __forceinline__ V add(V a, V b) { int s = a + b; return s > Q ? Q : s; }
    __device__ static __forceinline__ uint32_t key(V v) { return (uint32_t)v; }
    __device__ static __forceinline__ V from_key(uint32_t k) { return (int)k; }
    __device__ static __forceinline__ V zero() { return 0; }
    __device__ static __forceinline__ V big() { return 0x7FFFFFFF; }
    __device__ static __forceinline__ uint32_t quant(float x)
    {
        float y = fminf(fmaxf(x * 32.0f, -32767.0f), 32767.0f);
        return (uint32_t)__float2int_rn(y) & 0xFFFFu;
    }
    __device__ static __forceinline__ float to_float(V v) { return (float)v; }
    __device__ static __forceinline__ V sub(V a, V b) { return a - b; }
    __device__ static __forceinline__ V f1(V a, V b)
    {
        const V m = min(a < 0 ? -a : a, b < 0 ? -b : b);
        return ((a < 0) != (b < 0)) ? -m : m;
    }
    __device__ static __forceinline__ V g1(V a, V b, uint32_t s)
    {
        const V x = (s ? -a : a) + b;
        return x > Q ? Q : (x < -Q ? -Q : x);
    }
};

struct QI8 {
    static constexpr int EPW = 4, BITS = 8, FIXED = 1, Q = 127, FRAC = 2, VBITS = 7;
    typedef int V;
    __device__ static __forceinline__ uint32_t F(uint32_t a, uint32_t b)
    {
        uint32_t m = __vminu4(__vabsss4(a), __vabsss4(b));
        uint32_t mask = (((a ^ b) & 0x80808080u) >> 7) * 0xFFu;
        return (m & ~mask) | (__vneg4(m) & mask);
    }
    // s: bits 0..3 = partial sums of the four elements
    __device__ static __forceinline__ uint32_t G(uint32_t a, uint32_t b, uint32_t s)
    {
        uint32_t mask = (((s & 15u) * 0x00204081u) & 0x01010101u) * 0xFFu;
        uint32_t na = (a & ~mask) | (__vneg4(a) & mask);
        return __vmaxs4(__vaddss4(na, b), 0x81818181u);  // saturate to [-Q, Q]
    }
    __device__ static __forceinline__ V elem(uint32_t w, int k) { return (int)(int8_t)(w >> (8 * k)); }
    __device__ static __forceinline__ V absv(V v) { return v < 0 ? -v : v; }
    __device__ static __forceinline__ V add(V a, V b) { int s = a + b; return s > Q ? Q : s; }
    __device__ static __forceinline__ uint32_t key(V v) { return (uint32_t)v; }
    __device__ static __forceinline__ V from_key(uint32_t k) { return (int)k; }
    __device__ static __forceinline__ V zero() { return 0; }
    __device__ static __forceinline__ V big() { return 0x7FFFFFFF; }
    __device__ static __forceinline__ uint32_t quant(float x)
    {
        float y = fminf(fmaxf(x * 4.0f, -127.0f), 127.0f);
        return (uint32_t)__float2int_rn(y) & 0xFFu;
    }
    __device__ static __forceinline__ float to_float(V v) { return (float)v; }
    __device__ static __forceinline__ V sub(V a, V b) { return a - b; }
    __device__ static __forceinline__ V f1(V a, V b)
    {
        const V m = min(a < 0 ? -a : a, b < 0 ? -b : b);
        return ((a < 0) != (b < 0)) ? -m : m;
    }
    __device__ static __forceinline__ V g1(V a, V b, uint32_t s)
    {
        const V x = (s ? -a : a) + b;
        return x > Q ? Q : (x < -Q ? -Q : x);
    }
};

// ---------------------------------------------------------------------------
// Warp context
struct Ctx {
    const Item *P;   // the current task's item (shared-memory copy)
    char *sm;        // warp's shared slice
    char *gm;        // warp's global scratch slice
    int lane, L, seg, slot, fpw, fiw;
    int N, n;
    int n_active;    // warp-uniform
    const uint32_t *ops;
    int n_ops;
    uint32_t idxL[2], idxS[2];  // per-layer slot tables: layers 1..12, 6 x 5 bits per word
#ifdef PSCL_OPPROF
    unsigned long long *prof;   // step-profiling builds: cycle and step counters
#endif
};

#ifdef PSCL_OPPROF
// step-profiling builds: lane 0 adds a step's SM cycles to its category
// (0..6 opcodes, 7 + node type for OP_NODE, 12 frame loading, 13 the final
// CRC selection and output; 14 counts the two-candidate selections that
// took the general path, inside the steps above)
__device__ __forceinline__ void prof_add(const Ctx &c, int cat, long long t0)
{
    __syncwarp();
    if (c.lane == 0 && c.prof) {
        atomicAdd(&c.prof[2 * cat], (unsigned long long)(clock64() - t0));
        atomicAdd(&c.prof[2 * cat + 1], 1ull);
    }
}
#define PSCL_PROF_T0(v) const long long v = clock64()
#define PSCL_PROF_ADD(cat, v) prof_add(c, cat, v)
#else
#define PSCL_PROF_T0(v)
#define PSCL_PROF_ADD(cat, v)
#endif

// slot of layer d (1 <= d <= kTabLayers) in a table
__device__ __forceinline__ int tab_get(const uint32_t (&t)[2], int d)
{
    const int e = d - 1;
    uint32_t w = e < 6 ? t[0] : t[1];
    int sh = 5 * (e < 6 ? e : e - 6);
    return (int)((w >> sh) & 31u);
}
__device__ __forceinline__ void tab_set(uint32_t (&t)[2], int d, int v)
{
    const int e = d - 1;
    int sh = 5 * (e < 6 ? e : e - 6);
    uint32_t m = ~(31u << sh);
    if (e < 6) t[0] = (t[0] & m) | ((uint32_t)v << sh);
    else t[1] = (t[1] & m) | ((uint32_t)v << sh);
}
__device__ __forceinline__ void tab_fill(uint32_t (&t)[2], int v)
{
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < 6; ++k) w |= (uint32_t)v << (5 * k);
    t[0] = w;
    t[1] = w;
}

#ifdef PSCL_CHECKED
__device__ __forceinline__ bool chk(const Ctx &c, bool ok, uint32_t code)
{
    if (!ok) atomicOr(c.P->err, code);
    return ok;
}
#define PSCL_OK_IDX(c, idx, cap, code) chk(c, (uint32_t)(idx) < (uint32_t)(cap), code)
#else
#define PSCL_OK_IDX(c, idx, cap, code) true
#endif

// Base pointers of every buffer of the warp, computed once per item and kept
// in a small table behind the item copy: [0..11] LLR layers, [12..23] BL,
// [24..35] BR.
__device__ __forceinline__ uint32_t **ptab(const Ctx &c) { return (uint32_t **)(c.sm + kItemBytes); }
__device__ __forceinline__ uint32_t *llr_layer(const Ctx &c, int d) { return ptab(c)[d]; }
__device__ __forceinline__ uint32_t *bl_layer(const Ctx &c, int d) { return ptab(c)[kMaxLayers + d]; }
__device__ __forceinline__ uint32_t *br_layer(const Ctx &c, int d) { return ptab(c)[2 * kMaxLayers + d]; }

// LLR layers store the words of a path in groups of four: word w of column
// col sits at ((w / 4) * width + col) * 4 + w % 4, so a lane moves four
// consecutive words with one 16-byte access and a warp row is 512 bytes.
__device__ __forceinline__ int qa(int w, int col, int width) { return (((w >> 2) * width + col) << 2) + (w & 3); }

__device__ __forceinline__ uint32_t ld(const Ctx &c, const uint32_t *p, int idx, uint32_t cap, uint32_t code)
{
    if (!PSCL_OK_IDX(c, idx, cap, code)) return 0u;
    return p[idx];
}
__device__ __forceinline__ void st(const Ctx &c, uint32_t *p, int idx, uint32_t cap, uint32_t v, uint32_t code)
{
    if (!PSCL_OK_IDX(c, idx, cap, code)) return;
    p[idx] = v;
}
// quad q of column col (16-byte aligned)
__device__ __forceinline__ uint4 ld4(const Ctx &c, const uint32_t *p, int q, int col, int width, uint32_t cap,
                                     uint32_t code)
{
    const int idx = (q * width + col) << 2;
    if (!PSCL_OK_IDX(c, idx + 3, cap, code)) return make_uint4(0u, 0u, 0u, 0u);
    return *reinterpret_cast<const uint4 *>(p + idx);
}
__device__ __forceinline__ void st4(const Ctx &c, uint32_t *p, int q, int col, uint32_t cap, uint4 v, uint32_t code)
{
    const int idx = (q * 32 + col) << 2;
    if (!PSCL_OK_IDX(c, idx + 3, cap, code)) return;
    *reinterpret_cast<uint4 *>(p + idx) = v;
}

__device__ __forceinline__ uint64_t shfl64(uint64_t v, int src)
{
    uint32_t lo = __shfl_sync(PSCL_FULL, (uint32_t)v, src);
    uint32_t hi = __shfl_sync(PSCL_FULL, (uint32_t)(v >> 32), src);
    return ((uint64_t)hi << 32) | lo;
}
__device__ __forceinline__ uint64_t shfl64_xor(uint64_t v, int m)
{
    uint32_t lo = __shfl_xor_sync(PSCL_FULL, (uint32_t)v, m);
    uint32_t hi = __shfl_xor_sync(PSCL_FULL, (uint32_t)(v >> 32), m);
    return ((uint64_t)hi << 32) | lo;
}

// words w0..w0+3 of a column (w0 a multiple of 4), one 16-byte access when
// all four exist
__device__ __forceinline__ void fetch4(const Ctx &c, const uint32_t *p, int w0, int nw, int col, int width,
                                       uint32_t cap, uint32_t (&out)[4])
{
    if (nw - w0 >= 4) {
        const uint4 v = ld4(c, p, w0 >> 2, col, width, cap, 1u);
        out[0] = v.x;
        out[1] = v.y;
        out[2] = v.z;
        out[3] = v.w;
    } else {
#pragma unroll
        for (int k = 0; k < 4; ++k) out[k] = w0 + k < nw ? ld(c, p, qa(w0 + k, col, width), cap, 1u) : 0u;
    }
}

// ---------------------------------------------------------------------------
// f step at depth d: layer d+1 (own column) = f(layer d) for the left child.
// Slots without an active path skip the memory traffic (their columns are
// never read before being rewritten).
template <class Qt>
__device__ __forceinline__ void op_f(Ctx &c, int d)
{
    const int S = c.N >> d, H = S >> 1;
    const uint32_t *in = llr_layer(c, d);
    uint32_t *out = llr_layer(c, d + 1);
    const uint32_t cap_in = c.P->lay.llr_words[d], cap_out = c.P->lay.llr_words[d + 1];
    const int win = d == 0 ? c.fpw : 32;
    const int cin = d == 0 ? c.fiw : c.seg + tab_get(c.idxL, d);
    const bool act = c.slot < c.n_active;
    if (act) {
        if (H >= 4 * Qt::EPW) {
            const int HQ = H / (4 * Qt::EPW);
            // blocks of four quad pairs: all eight loads are issued before
            // any store (the buffers could alias as far as the compiler
            // knows, so it would not hoist them itself)
            constexpr int U = 4;
            int q = 0;
            for (; q + U <= HQ; q += U) {
                uint4 a[U], b[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    a[u] = ld4(c, in, q + u, cin, win, cap_in, 1u);
                    b[u] = ld4(c, in, q + u + HQ, cin, win, cap_in, 1u);
                }
#pragma unroll
                for (int u = 0; u < U; ++u)
                    st4(c, out, q + u, c.lane, cap_out,
                        make_uint4(Qt::F(a[u].x, b[u].x), Qt::F(a[u].y, b[u].y), Qt::F(a[u].z, b[u].z),
                                   Qt::F(a[u].w, b[u].w)),
                        2u);
            }
            for (; q < HQ; ++q) {
                const uint4 a = ld4(c, in, q, cin, win, cap_in, 1u);
                const uint4 b = ld4(c, in, q + HQ, cin, win, cap_in, 1u);
                st4(c, out, q, c.lane, cap_out,
                    make_uint4(Qt::F(a.x, b.x), Qt::F(a.y, b.y), Qt::F(a.z, b.z), Qt::F(a.w, b.w)), 2u);
            }
        } else if (H >= Qt::EPW) {
            const int HW = H / Qt::EPW;
            for (int w = 0; w < HW; ++w) {
                const uint32_t a = ld(c, in, qa(w, cin, win), cap_in, 1u);
                const uint32_t b = ld(c, in, qa(w + HW, cin, win), cap_in, 1u);
                st(c, out, qa(w, c.lane, 32), cap_out, Qt::F(a, b), 2u);
            }
        } else {
            const uint32_t wd = ld(c, in, qa(0, cin, win), cap_in, 1u);
            st(c, out, qa(0, c.lane, 32), cap_out, Qt::F(wd, wd >> (H * Qt::BITS)), 2u);
        }
    }
    tab_set(c.idxL, d + 1, c.slot);
}

// g step at depth d: layer d+1 (own column) = g(layer d, beta of the left
// child, stored in BL_{d+1}).
template <class Qt>
__device__ __forceinline__ void op_g(Ctx &c, int d)
{
    const int S = c.N >> d, H = S >> 1;
    const uint32_t *in = llr_layer(c, d);
    uint32_t *out = llr_layer(c, d + 1);
    const uint32_t *bl = bl_layer(c, d + 1);
    const uint32_t cap_in = c.P->lay.llr_words[d], cap_out = c.P->lay.llr_words[d + 1];
    const uint32_t cap_b = c.P->lay.b_words[d + 1];
    const int win = d == 0 ? c.fpw : 32;
    const int cin = d == 0 ? c.fiw : c.seg + tab_get(c.idxL, d);
    const int cs = c.seg + tab_get(c.idxS, d + 1);
    const bool act = c.slot < c.n_active;
    constexpr uint32_t M1 = (1u << Qt::EPW) - 1u;
    if (act) {
        if (H >= 4 * Qt::EPW) {
            const int HQ = H / (4 * Qt::EPW);
            constexpr int QPB = 32 / (4 * Qt::EPW);  // quads per 32-bit beta word
            auto sbits = [&](int q) {
                const uint32_t bw = ld(c, bl, (q / QPB) * 32 + cs, cap_b, 4u);
                return bw >> ((q % QPB) * 4 * Qt::EPW);
            };
            auto gq = [&](const uint4 &a, const uint4 &b, uint32_t sb) {
                return make_uint4(Qt::G(a.x, b.x, sb & M1), Qt::G(a.y, b.y, (sb >> Qt::EPW) & M1),
                                  Qt::G(a.z, b.z, (sb >> (2 * Qt::EPW)) & M1),
                                  Qt::G(a.w, b.w, (sb >> (3 * Qt::EPW)) & M1));
            };
            constexpr int U = 4;
            int q = 0;
            for (; q + U <= HQ; q += U) {
                uint4 a[U], b[U];
                uint32_t sb[U];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    a[u] = ld4(c, in, q + u, cin, win, cap_in, 1u);
                    b[u] = ld4(c, in, q + u + HQ, cin, win, cap_in, 1u);
                    sb[u] = sbits(q + u);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) st4(c, out, q + u, c.lane, cap_out, gq(a[u], b[u], sb[u]), 2u);
            }
            for (; q < HQ; ++q) {
                const uint4 a = ld4(c, in, q, cin, win, cap_in, 1u);
                const uint4 b = ld4(c, in, q + HQ, cin, win, cap_in, 1u);
                st4(c, out, q, c.lane, cap_out, gq(a, b, sbits(q)), 2u);
            }
        } else if (H >= Qt::EPW) {
            const int HW = H / Qt::EPW;
            const uint32_t bw = ld(c, bl, cs, cap_b, 4u);
            for (int w = 0; w < HW; ++w) {
                const uint32_t a = ld(c, in, qa(w, cin, win), cap_in, 1u);
                const uint32_t b = ld(c, in, qa(w + HW, cin, win), cap_in, 1u);
                st(c, out, qa(w, c.lane, 32), cap_out, Qt::G(a, b, (bw >> (w * Qt::EPW)) & M1), 2u);
            }
        } else {
            const uint32_t wd = ld(c, in, qa(0, cin, win), cap_in, 1u);
            const uint32_t sb = ld(c, bl, cs, cap_b, 4u) & ((1u << H) - 1u);
            st(c, out, qa(0, c.lane, 32), cap_out, Qt::G(wd, wd >> (H * Qt::BITS), sb), 2u);
        }
    }
    tab_set(c.idxL, d + 1, c.slot);
}

// h step: the right child at depth d is complete (its beta in BR_d); the
// parent's beta (BL_d ^ BR_d, BR_d) goes to BL_{d-1} (parent is a left
// child) or BR_{d-1}.
__device__ __forceinline__ void op_comb(Ctx &c, int d, int parent_side)
{
    const int S = c.N >> d;
    const uint32_t *bl = bl_layer(c, d);
    const uint32_t *br = br_layer(c, d);
    uint32_t *dst = parent_side == 0 ? bl_layer(c, d - 1) : br_layer(c, d - 1);
    const uint32_t cap = c.P->lay.b_words[d], capd = c.P->lay.b_words[d - 1];
    const int cl = c.seg + tab_get(c.idxS, d);
    if (S >= 32) {
        const int W = S >> 5;
        int w = 0;
        for (; w + 4 <= W; w += 4) {  // loads first: the buffers could alias for the compiler
            uint32_t l[4], r[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                l[u] = ld(c, bl, (w + u) * 32 + cl, cap, 8u);
                r[u] = ld(c, br, (w + u) * 32 + c.lane, cap, 8u);
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                st(c, dst, (w + u) * 32 + c.lane, capd, l[u] ^ r[u], 16u);
                st(c, dst, (w + u + W) * 32 + c.lane, capd, r[u], 16u);
            }
        }
        for (; w < W; ++w) {
            uint32_t l = ld(c, bl, w * 32 + cl, cap, 8u);
            uint32_t r = ld(c, br, w * 32 + c.lane, cap, 8u);
            st(c, dst, w * 32 + c.lane, capd, l ^ r, 16u);
            st(c, dst, (w + W) * 32 + c.lane, capd, r, 16u);
        }
    } else {
        const uint32_t m = (1u << S) - 1u;
        uint32_t l = ld(c, bl, cl, cap, 8u);
        uint32_t r = ld(c, br, c.lane, cap, 8u) & m;
        st(c, dst, c.lane, capd, ((l ^ r) & m) | (r << S), 16u);
    }
    if (parent_side == 0) tab_set(c.idxS, d - 1, c.slot);
}

// ---------------------------------------------------------------------------
// Balanced pairwise sum over index order, fed one element at a time: the
// binary-counter form adds acc[l] + v exactly where the recursive tree
// s(lo, hi) = s(lo, mid) + s(mid, hi) would.  Returns the value stored at the
// last push (the full sum after the last element of a power-of-two run).
template <class Qt>
struct TreeSum {
    typename Qt::V acc[kMaxLayers];
    __device__ __forceinline__ typename Qt::V push(typename Qt::V v, int i)
    {
#pragma unroll
        for (int l = 0; l < kMaxLayers; ++l) {
            if ((i >> l) & 1) {
                v = Qt::add(acc[l], v);
            } else {
                acc[l] = v;
                return v;
            }
        }
        return v;
    }
};

// segment-wide minimum of the metrics of active slots (fixed point only)
template <class Qt>
__device__ __forceinline__ void normalise(Ctx &c, typename Qt::V &pm)
{
    if (!Qt::FIXED) return;
    typename Qt::V v = c.slot < c.n_active ? pm : Qt::big();
    if (c.L == 32) {
        v = (typename Qt::V)__reduce_min_sync(PSCL_FULL, (int)v);
    } else {
        for (int m = 1; m < c.L; m <<= 1) {
            typename Qt::V o = __shfl_xor_sync(PSCL_FULL, v, m);
            v = o < v ? o : v;
        }
    }
    pm = Qt::sub(pm, v);
}

// Bitonic sort (ascending) of the L*M keys of a segment; element e = slot*M + m.
template <int M>
__device__ __forceinline__ void bitonic_seg(uint32_t (&k)[M], int L, int slot)
{
    const int E = L * M;
    for (int size = 2; size <= E; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            if (stride >= M) {
                const int ls = stride / M;
                const bool lower = (slot & ls) == 0;
#pragma unroll
                for (int m = 0; m < M; ++m) {
                    const int e = slot * M + m;
                    const bool up = (e & size) == 0;
                    const uint32_t o = __shfl_xor_sync(PSCL_FULL, k[m], ls);
                    k[m] = lower == up ? min(o, k[m]) : max(o, k[m]);
                }
            } else {
#pragma unroll
                for (int sb = 0; (1 << sb) < M; ++sb) {
                    if (stride == (1 << sb)) {
#pragma unroll
                        for (int m = 0; m < M; ++m) {
                            if ((m & (1 << sb)) == 0) {
                                const int mp = m | (1 << sb);
                                const int e = slot * M + m;
                                const bool up = (e & size) == 0;
                                const uint32_t lo = min(k[m], k[mp]), hi = max(k[m], k[mp]);
                                k[m] = up ? lo : hi;
                                k[mp] = up ? hi : lo;
                            }
                        }
                    }
                }
            }
        }
    }
}

// Keep the min(L, n_active*M) smallest (PM, c) candidates, c = slot*M + m,
// and give them new slots in increasing c.  kp[m] is the ordered bit pattern
// of candidate m's metric.  On return, lanes with slot < n_keep know their
// parent slot, candidate index and metric key.  The L-th smallest metric
// value tau is found first (float: a 32-bit bitonic network of the keys;
// fixed point: bisection on the metric's bits with ballot counts); every
// candidate below tau survives, and of those equal to tau the first in
// candidate order fill the remaining places.
template <int M, int VBITS>
__device__ __forceinline__ void select_paths(Ctx &c, const uint32_t (&kp)[M], int &par, int &cand,
                                             uint32_t &newkey, int &n_keep, bool &ident)
{
    ident = false;
    const int na = c.n_active, L = c.L;
    const int n_cand = na * M;
    if (n_cand <= L) {
        n_keep = n_cand;
        par = c.slot < n_keep ? c.slot / M : 0;
        cand = c.slot < n_keep ? c.slot % M : 0;
        uint32_t v = 0;
#pragma unroll
        for (int m = 0; m < M; ++m) {
            uint32_t x = __shfl_sync(PSCL_FULL, kp[m], c.seg + par);
            if (m == cand) v = x;
        }
        newkey = v;
        return;
    }
    n_keep = L;
    if (na == L) {
        // every path's first candidate ranks before every other candidate:
        // the first candidates survive in place, nothing is sorted
        uint32_t mn = 0xFFFFFFFFu;
#pragma unroll
        for (int m = 1; m < M; ++m) mn = min(mn, kp[m]);
        const uint32_t mx = __reduce_max_sync(PSCL_FULL, kp[0]);
        mn = __reduce_min_sync(PSCL_FULL, mn);
        if (mn > mx) {
            par = c.slot;
            cand = 0;
            newkey = kp[0];
            ident = true;
            return;
        }
    }
    const uint32_t segmask = L == 32 ? 0xFFFFFFFFu : (((1u << L) - 1u) << c.seg);
    uint32_t a[M];
#pragma unroll
    for (int m = 0; m < M; ++m) a[m] = c.slot < na ? kp[m] : 0xFFFFFFFFu;
    uint32_t tau;
    if constexpr (VBITS > 0) {
        uint32_t v = 0;
#pragma unroll 1
        for (int bit = VBITS - 1; bit >= 0; --bit) {
            const uint32_t cv = v | ((1u << bit) - 1u);
            int cnt = 0;
#pragma unroll
            for (int m = 0; m < M; ++m) cnt += __popc(__ballot_sync(PSCL_FULL, a[m] <= cv) & segmask);
            if (cnt < L) v |= 1u << bit;
        }
        tau = v;
    } else {
        uint32_t k[M];
#pragma unroll
        for (int m = 0; m < M; ++m) k[m] = a[m];
        bitonic_seg<M>(k, L, c.slot);
        const int tp = (L - 1) / M, tm = (L - 1) % M;
        uint32_t mine = 0;
#pragma unroll
        for (int m = 0; m < M; ++m)
            if (m == tm) mine = k[m];
        tau = __shfl_sync(PSCL_FULL, mine, c.seg + tp);
    }
    const uint32_t lt = ((1u << c.lane) - 1u) & segmask;
    int n_less = 0, eq_rank = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        n_less += __popc(__ballot_sync(PSCL_FULL, a[m] < tau) & segmask);
        eq_rank += __popc(__ballot_sync(PSCL_FULL, a[m] == tau) & lt);
    }
    const int need = L - n_less;
    bool surv[M];
    int r = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) {
        const bool eq = a[m] == tau;
        surv[m] = a[m] < tau || (eq && eq_rank < need);
        eq_rank += eq ? 1 : 0;
        r += __popc(__ballot_sync(PSCL_FULL, surv[m]) & lt);
    }
    uint32_t *src = (uint32_t *)(c.sm + c.P->lay.src_off);
#pragma unroll
    for (int m = 0; m < M; ++m) {
        if (surv[m]) {
            if (PSCL_OK_IDX(c, c.seg + r, 32, 32u)) {
                src[2 * (c.seg + r)] = ((uint32_t)c.slot << 8) | (uint32_t)m;
                src[2 * (c.seg + r) + 1] = kp[m];
            }
            ++r;
        }
    }
    __syncwarp();
    const uint32_t e0 = src[2 * c.lane], e1 = src[2 * c.lane + 1];
    __syncwarp();
    par = (int)(e0 >> 8) & (c.L - 1);
    cand = (int)(e0 & 255u);
    if (cand >= M) cand = 0;
    newkey = e1;
}

// The general case of select_m2: the L-th smallest metric value is found
// (float: 32-bit bitonic network of the 2L patterns; fixed point: bisection on
// the metric's bits with ballot counts) and ties at that value are resolved in
// candidate order; the survivors are scattered through shared memory (src, 64
// words) into their new slots.  Returns (key << 32) | (parent slot << 8) |
// candidate.  The node-capable kernel calls it out of line (its register
// pressure is highest around the node handlers).
template <int VBITS>
__device__ __forceinline__ uint64_t select_m2_general(uint32_t a, uint32_t b, uint32_t ka, uint32_t kb, int L,
                                                      int lane, int slot, int seg, uint32_t *src)
{
    const uint32_t segmask = L == 32 ? 0xFFFFFFFFu : (((1u << L) - 1u) << seg);
    uint32_t tau;
    if constexpr (VBITS > 0) {
        // fixed point: metrics are integers below 2^VBITS, so the L-th
        // smallest value is found by bisection on its bits (ballot counts)
        uint32_t v = 0;
#pragma unroll
        for (int bit = VBITS - 1; bit >= 0; --bit) {
            const uint32_t cand = v | ((1u << bit) - 1u);
            const int cnt = __popc(__ballot_sync(PSCL_FULL, a <= cand) & segmask) +
                            __popc(__ballot_sync(PSCL_FULL, b <= cand) & segmask);
            if (cnt < L) v |= 1u << bit;
        }
        tau = v;
    } else {
        // float: bitonic sort of the 2L metric patterns, element e = 2*slot + m
        uint32_t k0 = a, k1 = b;
        for (int size = 2; size <= 2 * L; size <<= 1) {
            const bool up = ((slot << 1) & size) == 0;
            for (int stride = size >> 1; stride > 0; stride >>= 1) {
                if (stride == 1) {
                    const uint32_t lo = min(k0, k1), hi = max(k0, k1);
                    k0 = up ? lo : hi;
                    k1 = up ? hi : lo;
                } else {
                    const int ls = stride >> 1;
                    const bool takemin = ((slot & ls) == 0) == up;
                    const uint32_t o0 = __shfl_xor_sync(PSCL_FULL, k0, ls);
                    const uint32_t o1 = __shfl_xor_sync(PSCL_FULL, k1, ls);
                    k0 = takemin ? min(k0, o0) : max(k0, o0);
                    k1 = takemin ? min(k1, o1) : max(k1, o1);
                }
            }
        }
        const int tp = (L - 1) >> 1;
        const uint32_t tsel = ((L - 1) & 1) ? k1 : k0;
        tau = __shfl_sync(PSCL_FULL, tsel, seg + tp);
    }
    const uint32_t lt = ((1u << lane) - 1u) & segmask;
    const uint32_t BA = __ballot_sync(PSCL_FULL, a < tau) & segmask;
    const uint32_t BB = __ballot_sync(PSCL_FULL, b < tau) & segmask;
    const uint32_t EA = __ballot_sync(PSCL_FULL, a == tau) & segmask;
    const uint32_t EB = __ballot_sync(PSCL_FULL, b == tau) & segmask;
    const int need = L - __popc(BA) - __popc(BB);
    const int ra = __popc(EA & lt) + __popc(EB & lt);
    const bool sa = a < tau || (a == tau && ra < need);
    const int rb = ra + (a == tau ? 1 : 0);
    const bool sb = b < tau || (b == tau && rb < need);
    const uint32_t SA = __ballot_sync(PSCL_FULL, sa) & segmask;
    const uint32_t SB = __ballot_sync(PSCL_FULL, sb) & segmask;
    int r = __popc(SA & lt) + __popc(SB & lt);
    if (sa) {
        src[2 * (seg + r)] = (uint32_t)slot << 8;
        src[2 * (seg + r) + 1] = ka;
        ++r;
    }
    if (sb) {
        src[2 * (seg + r)] = ((uint32_t)slot << 8) | 1u;
        src[2 * (seg + r) + 1] = kb;
    }
    __syncwarp();
    const uint32_t e0 = src[2 * lane], e1 = src[2 * lane + 1];
    __syncwarp();
    return ((uint64_t)e1 << 32) | e0;
}
template <int VBITS>
__device__ __noinline__ uint64_t select_m2_general_call(uint32_t a, uint32_t b, uint32_t ka, uint32_t kb, int L,
                                                        int lane, int slot, int seg, uint32_t *src)
{
    return select_m2_general<VBITS>(a, b, ka, kb, L, lane, slot, seg, src);
}

// Two candidates per path (an information leaf, or a REP node): candidate
// (p, 0) has metric key ka, (p, 1) key kb, candidate ids c = 2p and 2p + 1.
// Same result as select_paths<2>: the L smallest (PM, c) survive and take new
// slots in increasing c.  When every path's second candidate ranks after
// every first candidate, the first candidates are the survivors and no sort
// is needed; otherwise the L-th smallest metric value is found with a 32-bit
// bitonic network and ties at that value are resolved in candidate order.
template <int VBITS, bool OUT>
__device__ __forceinline__ void select_m2(Ctx &c, uint32_t ka, uint32_t kb, int &par, int &cand,
                                          uint32_t &newkey, int &n_keep, bool &ident)
{
    const int na = c.n_active, L = c.L;
    ident = false;
    if (2 * na <= L) {
        n_keep = 2 * na;
        const bool live = c.slot < n_keep;
        par = live ? c.slot >> 1 : 0;
        cand = live ? c.slot & 1 : 0;
        const uint32_t x0 = __shfl_sync(PSCL_FULL, ka, c.seg + par);
        const uint32_t x1 = __shfl_sync(PSCL_FULL, kb, c.seg + par);
        newkey = cand ? x1 : x0;
        return;
    }
    n_keep = L;
    const bool act = c.slot < na;
    const uint32_t a = act ? ka : 0xFFFFFFFFu, b = act ? kb : 0xFFFFFFFFu;
    if (na == L) {
        // warp-wide reductions (one instruction each): when every flip
        // candidate of the warp ranks after every keep candidate, each frame
        // of the warp keeps its paths in place (a sufficient condition per
        // frame, and the same decision in every lane)
        const uint32_t mx = __reduce_max_sync(PSCL_FULL, a);
        const uint32_t mn = __reduce_min_sync(PSCL_FULL, b);
        if (mn > mx) {
            par = c.slot;
            cand = 0;
            newkey = ka;
            ident = true;
            return;
        }
    }
    uint32_t *src = (uint32_t *)(c.sm + c.P->lay.src_off);
    PSCL_PROF_T0(t_sel);
    const uint64_t r = OUT ? select_m2_general_call<VBITS>(a, b, ka, kb, L, c.lane, c.slot, c.seg, src)
                           : select_m2_general<VBITS>(a, b, ka, kb, L, c.lane, c.slot, c.seg, src);
    PSCL_PROF_ADD(14, t_sel);
    const uint32_t e0 = (uint32_t)r, e1 = (uint32_t)(r >> 32);
    par = (int)(e0 >> 8) & (L - 1);
    cand = (int)(e0 & 1u);
    newkey = e1;
}

// ---------------------------------------------------------------------------
// A leaf or pruned node at depth d (Sec. II-B; candidate rules as in the
// header notes of the oracle and the ABI).
template <class Qt, int M>
__device__ __forceinline__ void node_select_finish(Ctx &c, int d, int type, int side, int t,
                                                   const uint32_t (&kp)[M], uint32_t h,
                                                   const uint32_t (&rp)[3], typename Qt::V &pm)
{
    const int S = c.N >> d;
    uint32_t *dst = side == 0 ? bl_layer(c, d) : br_layer(c, d);
    const uint32_t capd = c.P->lay.b_words[d];
    int par, cand, n_keep;
    uint32_t newkey;
    bool ident;
    if constexpr (M == 2) select_m2<Qt::VBITS, true>(c, kp[0], kp[1], par, cand, newkey, n_keep, ident);
    else select_paths<M, Qt::VBITS>(c, kp, par, cand, newkey, n_keep, ident);
    const int pl = c.seg + par;
    uint32_t hp = h, r0 = rp[0], r1 = rp[1], r2 = rp[2];
    if (!ident) {
        // the new path inherits its parent's slot tables (lazy copy)
        c.idxL[0] = __shfl_sync(PSCL_FULL, c.idxL[0], pl);
        c.idxL[1] = __shfl_sync(PSCL_FULL, c.idxL[1], pl);
        c.idxS[0] = __shfl_sync(PSCL_FULL, c.idxS[0], pl);
        c.idxS[1] = __shfl_sync(PSCL_FULL, c.idxS[1], pl);
        hp = __shfl_sync(PSCL_FULL, h, pl);
        r0 = __shfl_sync(PSCL_FULL, rp[0], pl);
        r1 = __shfl_sync(PSCL_FULL, rp[1], pl);
        r2 = __shfl_sync(PSCL_FULL, rp[2], pl);
    }
    pm = Qt::from_key(newkey);
    if (type == NT_REP) {
        const uint32_t ones = S >= 32 ? 0xFFFFFFFFu : ((1u << S) - 1u);
        const int W = S >= 32 ? S >> 5 : 1;
        for (int w = 0; w < W; ++w) st(c, dst, w * 32 + c.lane, capd, cand ? ones : 0u, 64u);
    } else {
        // R1 / SPC: parent's hard decisions with the candidate's flips
        int j = cand;
        if (type == NT_SPC) {
            const int parity = S > 32 ? (int)((r2 >> 16) & 1u) : (__popc(hp) & 1);
            j = (cand << 1) | ((__popc((unsigned)cand) & 1) ^ parity);
        }
        uint32_t pos[5] = {r0 & 0xFFFFu, r0 >> 16, r1 & 0xFFFFu, r1 >> 16, r2 & 0xFFFFu};
        if (S <= 32) {
            uint32_t b = hp;
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (k < t && ((j >> k) & 1)) b ^= 1u << (pos[k] & 31u);
            st(c, dst, c.lane, capd, b, 64u);
        } else if (ident) {
            // own hard decisions are already in place: apply the flips only
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if (k < t && ((j >> k) & 1)) {
                    const int w = (int)(pos[k] >> 5);
                    st(c, dst, w * 32 + c.lane, capd, ld(c, dst, w * 32 + c.lane, capd, 128u) ^ (1u << (pos[k] & 31u)),
                       64u);
                }
        } else {
            const int W = S >> 5;
            for (int w = 0; w < W; ++w) {
                uint32_t v = ld(c, dst, w * 32 + pl, capd, 128u);
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 5; ++k)
                    if (k < t && ((j >> k) & 1) && (int)(pos[k] >> 5) == w) v ^= 1u << (pos[k] & 31u);
                st(c, dst, w * 32 + c.lane, capd, v, 64u);
                __syncwarp();
            }
        }
    }
    if (side == 0) tab_set(c.idxS, d, c.slot);
    c.n_active = n_keep;
    normalise<Qt>(c, pm);
}

template <class Qt>
__device__ __forceinline__ void op_node(Ctx &c, int d, int type, int side, int t, typename Qt::V &pm)
{
    typedef typename Qt::V V;
    const int S = c.N >> d;
    const uint32_t *in = llr_layer(c, d);
    const uint32_t cap_in = c.P->lay.llr_words[d];
    const int win = d == 0 ? c.fpw : 32;
    const int cin = d == 0 ? c.fiw : c.seg + tab_get(c.idxL, d);
    uint32_t *dst = side == 0 ? bl_layer(c, d) : br_layer(c, d);
    const uint32_t capd = c.P->lay.b_words[d];

    if (type == NT_R0 || type == NT_REP) {
        TreeSum<Qt> t0, t1;
        V p0 = Qt::zero(), p1 = Qt::zero();
        const int nw = (S + Qt::EPW - 1) / Qt::EPW;
        for (int w0 = 0; w0 < nw; w0 += 4) {
            uint32_t wq[4];
            fetch4(c, in, w0, nw, cin, win, cap_in, wq);
#pragma unroll
            for (int k4 = 0; k4 < 4; ++k4) {
#pragma unroll
                for (int e = 0; e < Qt::EPW; ++e) {
                    const int i = (w0 + k4) * Qt::EPW + e;
                    if (i < S) {
                        const V v = Qt::elem(wq[k4], e);
                        p0 = t0.push(v < 0 ? Qt::absv(v) : Qt::zero(), i);
                        if (type == NT_REP) p1 = t1.push(v > 0 ? Qt::absv(v) : Qt::zero(), i);
                    }
                }
            }
        }
        if (type == NT_R0) {
            pm = Qt::add(pm, p0);
            const int W = S >= 32 ? S >> 5 : 1;
            for (int w = 0; w < W; ++w) st(c, dst, w * 32 + c.lane, capd, 0u, 64u);
            if (side == 0) tab_set(c.idxS, d, c.slot);
            normalise<Qt>(c, pm);
            return;
        }
        uint32_t kp[2] = {Qt::key(Qt::add(pm, p0)), Qt::key(Qt::add(pm, p1))};
        uint32_t rp[3] = {0u, 0u, 0u};
        node_select_finish<Qt, 2>(c, d, type, side, t, kp, 0u, rp, pm);
        return;
    }

    // R1 / SPC: hard decisions, parity, and the t least reliable positions
    V bv[5];
    int bi[5];
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        bv[k] = Qt::big();
        bi[k] = 0;
    }
    uint32_t hword = 0, hlast = 0;
    int parity = 0;
    const int nw = (S + Qt::EPW - 1) / Qt::EPW;
    for (int w0 = 0; w0 < nw; w0 += 4) {
        uint32_t wq[4];
        fetch4(c, in, w0, nw, cin, win, cap_in, wq);
#pragma unroll
        for (int ee = 0; ee < 4 * Qt::EPW; ++ee) {
            const int e = ee % Qt::EPW;
            const int i = w0 * Qt::EPW + ee;
            if (i < S) {
                const V v = Qt::elem(wq[ee / Qt::EPW], e);
                const V a = Qt::absv(v);
                hword |= (uint32_t)(v < 0) << (i & 31);
                if (a < bv[4]) {
                    bool placed = false;
#pragma unroll
                    for (int k = 4; k >= 1; --k) {
                        if (!placed) {
                            if (a < bv[k - 1]) {
                                bv[k] = bv[k - 1];
                                bi[k] = bi[k - 1];
                            } else {
                                bv[k] = a;
                                bi[k] = i;
                                placed = true;
                            }
                        }
                    }
                    if (!placed) {
                        bv[0] = a;
                        bi[0] = i;
                    }
                }
                if ((i & 31) == 31 || i == S - 1) {
                    parity ^= __popc(hword) & 1;
                    if (S > 32) st(c, dst, (i >> 5) * 32 + c.lane, capd, hword, 64u);
                    hlast = hword;
                    hword = 0;
                }
            }
        }
    }
    uint32_t rp[3] = {(uint32_t)bi[0] | ((uint32_t)bi[1] << 16), (uint32_t)bi[2] | ((uint32_t)bi[3] << 16),
                      (uint32_t)bi[4] | ((uint32_t)parity << 16)};
    const uint32_t h = S <= 32 ? hlast : 0u;
    // candidate penalties: left fold over flipped ranks (ascending)
#define PSCL_CANDS(MM)                                                                   \
    {                                                                                    \
        uint32_t kp[MM];                                                                 \
        _Pragma("unroll") for (int m = 0; m < MM; ++m)                                   \
        {                                                                                \
            int j = type == NT_R1 ? m : ((m << 1) | ((__popc((unsigned)m) & 1) ^ parity)); \
            V pen = Qt::zero();                                                          \
            _Pragma("unroll") for (int k = 0; k < 5; ++k) if (k < t && ((j >> k) & 1)) pen = \
                Qt::add(pen, bv[k]);                                                     \
            kp[m] = Qt::key(Qt::add(pm, pen));                                           \
        }                                                                                \
        node_select_finish<Qt, MM>(c, d, type, side, t, kp, h, rp, pm);                 \
    }
    const int M = type == NT_R1 ? (1 << t) : (1 << (t - 1));
    switch (M) {
    case 1: PSCL_CANDS(1) break;
    case 2: PSCL_CANDS(2) break;
    case 4: PSCL_CANDS(4) break;
    default: PSCL_CANDS(8) break;
    }
#undef PSCL_CANDS
}

// A subtree of S leaves (S = 2..8) with no pruned node, decoded in
// registers: the f, g, h steps and leaf decisions of Algorithm 1 without
// touching memory.  a[] holds the node's LLRs.  fz: bit i set = leaf i
// frozen.  `shuf` moves the register state of the enclosing levels from a
// parent lane after a selection (the lazy path copy of the register part);
// when every path keeps its own slot nothing moves.  Returns the node's
// partial sums (S bits).
template <class Qt, int S, bool OUT, class Shuf>
__device__ __forceinline__ uint32_t rsub(Ctx &c, typename Qt::V (&a)[S], uint32_t fz, typename Qt::V &pm,
                                         const Shuf &shuf)
{
    typedef typename Qt::V V;
    if constexpr (S == 1) {
        const V lam = a[0];
        if (fz & 1u) {
            pm = Qt::add(pm, lam < 0 ? Qt::absv(lam) : Qt::zero());
            normalise<Qt>(c, pm);
            return 0u;
        }
        int par, cand, nk;
        uint32_t nkey;
        bool ident;
        select_m2<Qt::VBITS, OUT>(c, Qt::key(pm), Qt::key(Qt::add(pm, Qt::absv(lam))), par, cand, nkey, nk, ident);
        uint32_t hd = (uint32_t)(lam < 0);
        if (!ident) {
            const int pl = c.seg + par;
            c.idxL[0] = __shfl_sync(PSCL_FULL, c.idxL[0], pl);
            c.idxL[1] = __shfl_sync(PSCL_FULL, c.idxL[1], pl);
            c.idxS[0] = __shfl_sync(PSCL_FULL, c.idxS[0], pl);
            c.idxS[1] = __shfl_sync(PSCL_FULL, c.idxS[1], pl);
            hd = __shfl_sync(PSCL_FULL, hd, pl);
            shuf(pl);
        }
        pm = Qt::from_key(nkey);
        c.n_active = nk;
        normalise<Qt>(c, pm);
        return hd ^ (uint32_t)cand;
    } else {
        constexpr int H = S / 2;
        V l[H];
#pragma unroll
        for (int i = 0; i < H; ++i) l[i] = Qt::f1(a[i], a[i + H]);
        auto shuf_l = [&](int pl) {
            shuf(pl);
#pragma unroll
            for (int i = 0; i < S; ++i) a[i] = __shfl_sync(PSCL_FULL, a[i], pl);
        };
        uint32_t bl = rsub<Qt, H, OUT>(c, l, fz, pm, shuf_l);
        V r[H];
#pragma unroll
        for (int i = 0; i < H; ++i) r[i] = Qt::g1(a[i], a[i + H], (bl >> i) & 1u);
        auto shuf_r = [&](int pl) {
            shuf(pl);
            bl = __shfl_sync(PSCL_FULL, bl, pl);
        };
        const uint32_t br = rsub<Qt, H, OUT>(c, r, fz >> H, pm, shuf_r);
        const uint32_t m = (1u << H) - 1u;
        return ((bl ^ br) & m) | ((br & m) << H);
    }
}

template <class Qt, int S, bool OUT>
__device__ __forceinline__ void op_rsub(Ctx &c, int d, int side, uint32_t fz, typename Qt::V &pm)
{
    typedef typename Qt::V V;
    const uint32_t *in = llr_layer(c, d);
    const uint32_t cap = c.P->lay.llr_words[d];
    const int cin = c.seg + tab_get(c.idxL, d);
    V a[S];
    constexpr int NW = (S + Qt::EPW - 1) / Qt::EPW;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
        const uint32_t wd = ld(c, in, qa(w, cin, 32), cap, 1u);
#pragma unroll
        for (int e = 0; e < Qt::EPW; ++e)
            if (w * Qt::EPW + e < S) a[w * Qt::EPW + e] = Qt::elem(wd, e);
    }
    auto none = [](int) {};
    const uint32_t beta = rsub<Qt, S, OUT>(c, a, fz, pm, none);
    uint32_t *dst = side == 0 ? bl_layer(c, d) : br_layer(c, d);
    st(c, dst, c.lane, c.P->lay.b_words[d], beta, 64u);
    if (side == 0) tab_set(c.idxS, d, c.slot);
}

// Partial sums (S <= 16 bits) of a node finished in registers: into BL_d or
// BR_d, or, for a right child whose parent's h step is folded in (comb bit
// 0; parent side in bit 1), combined with the left sibling's partial sums
// (BL_d, the column the path holds) into BL/BR_{d-1}.
template <int S>
__device__ __forceinline__ void node_beta_out(Ctx &c, int d, int side, int comb, uint32_t beta)
{
    static_assert(S <= 16, "one 32-bit word for the parent");
    if (comb & 1) {
        constexpr uint32_t m2 = (1u << S) - 1u;
        const int psd = comb >> 1;
        const uint32_t sib = ld(c, bl_layer(c, d), c.seg + tab_get(c.idxS, d), c.P->lay.b_words[d], 8u);
        uint32_t *dst = psd == 0 ? bl_layer(c, d - 1) : br_layer(c, d - 1);
        st(c, dst, c.lane, c.P->lay.b_words[d - 1], ((sib ^ beta) & m2) | ((beta & m2) << S), 16u);
        if (psd == 0) tab_set(c.idxS, d - 1, c.slot);
        return;
    }
    uint32_t *dst = side == 0 ? bl_layer(c, d) : br_layer(c, d);
    st(c, dst, c.lane, c.P->lay.b_words[d], beta, 64u);
    if (side == 0) tab_set(c.idxS, d, c.slot);
}

// words of the node at depth d in the column the path holds (nw words)
template <int NW>
__device__ __forceinline__ void load_node(const Ctx &c, const uint32_t *in, int cin, uint32_t cap, uint32_t (&wd)[NW])
{
    if constexpr (NW >= 4) {
#pragma unroll
        for (int q = 0; q < NW / 4; ++q) {
            const uint4 v = ld4(c, in, q, cin, 32, cap, 1u);
            wd[4 * q] = v.x;
            wd[4 * q + 1] = v.y;
            wd[4 * q + 2] = v.z;
            wd[4 * q + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int w = 0; w < NW; ++w) wd[w] = ld(c, in, qa(w, cin, 32), cap, 1u);
    }
}

// An unpruned node of 2H leaves at depth d: the f step, the left subtree in
// registers, the g step (the node's LLRs read again from the column the path
// holds after the left half's selections), the right subtree in registers and
// the h step, with the left half's partial sums following the path through
// the right half's selections.  Equivalent to F, RSUB, G, RSUB, COMB.
template <class Qt, int H, bool OUT>
__device__ __forceinline__ void op_rsub2(Ctx &c, int d, int side, int comb, uint32_t fz, typename Qt::V &pm)
{
    typedef typename Qt::V V;
    constexpr int S = 2 * H;
    constexpr int NW = (S + Qt::EPW - 1) / Qt::EPW;
    const uint32_t *in = llr_layer(c, d);
    const uint32_t cap = c.P->lay.llr_words[d];
    uint32_t bl = 0u, br = 0u;
    auto carry = [&](int pl) { bl = __shfl_sync(PSCL_FULL, bl, pl); };
#pragma unroll 1
    for (int half = 0; half < 2; ++half) {
        uint32_t wd[NW];
        load_node<NW>(c, in, c.seg + tab_get(c.idxL, d), cap, wd);
        V a[H];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const V x = Qt::elem(wd[i / Qt::EPW], i % Qt::EPW);
            const V y = Qt::elem(wd[(i + H) / Qt::EPW], (i + H) % Qt::EPW);
            a[i] = half == 0 ? Qt::f1(x, y) : Qt::g1(x, y, (bl >> i) & 1u);
        }
        const uint32_t beta = rsub<Qt, H, OUT>(c, a, fz >> (half * H), pm, carry);
        if (half == 0) bl = beta;
        else br = beta;
    }
    constexpr uint32_t m = (1u << H) - 1u;
    node_beta_out<S>(c, d, side, comb, ((bl ^ br) & m) | ((br & m) << H));
}

// An unpruned node of 4H leaves (H = 4) at depth d, as four register
// subtrees of H leaves: for each quarter the node's LLRs are read again (at
// the column the path holds by then), the child's LLRs (f, or g with the
// left child's partial sums) and the grandchild's (f, or g with its left
// sibling's) are computed in registers, and the quarter is decoded.  The
// partial sums kept so far follow the paths through the selections.  Neither
// the children's nor the grandchildren's LLRs reach memory.  Equivalent to
// F, RSUB2, G, RSUB2, COMB.
template <class Qt, int H, bool OUT>
__device__ __forceinline__ void op_rsub4(Ctx &c, int d, int side, int comb, uint32_t fz, typename Qt::V &pm)
{
    typedef typename Qt::V V;
    constexpr int S = 4 * H, C = 2 * H;
    constexpr int NW = (S + Qt::EPW - 1) / Qt::EPW;
    constexpr uint32_t mh = (1u << H) - 1u, mc = (1u << C) - 1u;
    const uint32_t *in = llr_layer(c, d);
    const uint32_t cap = c.P->lay.llr_words[d];
    // b0: first grandchild; b1: first child (after the second quarter);
    // b2: third grandchild; b3: second child
    uint32_t b0 = 0u, b1 = 0u, b2 = 0u, b3 = 0u;
    auto carry = [&](int pl) {
        b0 = __shfl_sync(PSCL_FULL, b0, pl);
        b1 = __shfl_sync(PSCL_FULL, b1, pl);
        b2 = __shfl_sync(PSCL_FULL, b2, pl);
    };
#pragma unroll 1
    for (int q = 0; q < 4; ++q) {
        uint32_t wd[NW];
        load_node<NW>(c, in, c.seg + tab_get(c.idxL, d), cap, wd);
        const bool right_child = q >= 2, right_gc = (q & 1) != 0;
        const uint32_t sg = q < 2 ? b0 : b2;
        V l[H];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const V x0 = Qt::elem(wd[i / Qt::EPW], i % Qt::EPW);
            const V y0 = Qt::elem(wd[(i + C) / Qt::EPW], (i + C) % Qt::EPW);
            const V x1 = Qt::elem(wd[(i + H) / Qt::EPW], (i + H) % Qt::EPW);
            const V y1 = Qt::elem(wd[(i + H + C) / Qt::EPW], (i + H + C) % Qt::EPW);
            const V a0 = right_child ? Qt::g1(x0, y0, (b1 >> i) & 1u) : Qt::f1(x0, y0);
            const V a1 = right_child ? Qt::g1(x1, y1, (b1 >> (i + H)) & 1u) : Qt::f1(x1, y1);
            l[i] = right_gc ? Qt::g1(a0, a1, (sg >> i) & 1u) : Qt::f1(a0, a1);
        }
        const uint32_t beta = rsub<Qt, H, OUT>(c, l, fz >> (q * H), pm, carry);
        if (q == 0) b0 = beta;
        else if (q == 1) b1 = ((b0 ^ beta) & mh) | ((beta & mh) << H);
        else if (q == 2) b2 = beta;
        else b3 = ((b2 ^ beta) & mh) | ((beta & mh) << H);
    }
    node_beta_out<S>(c, d, side, comb, ((b1 ^ b3) & mc) | ((b3 & mc) << C));
}

// ---------------------------------------------------------------------------
// codeword word w (32 positions) of the lane's path (or of slot `col`'s path
// with its BL_1 column `cl`) once the root is complete
__device__ __forceinline__ uint32_t xhat_word(const Ctx &c, int w, int col, int cl)
{
    const Item &P = *c.P;
    if (P.root_special) return ld(c, br_layer(c, 0), w * 32 + col, P.lay.b_words[0], 256u);
    const int half = c.N >> 1;
    const uint32_t *bl = bl_layer(c, 1), *br = br_layer(c, 1);
    const uint32_t cap = P.lay.b_words[1];
    if (half >= 32) {
        const int W = half >> 5;
        if (w < W) return ld(c, bl, w * 32 + cl, cap, 256u) ^ ld(c, br, w * 32 + col, cap, 256u);
        return ld(c, br, (w - W) * 32 + col, cap, 256u);
    }
    const uint32_t m = (1u << half) - 1u;
    const uint32_t l = ld(c, bl, cl, cap, 256u), r = ld(c, br, col, cap, 256u) & m;
    return ((l ^ r) & m) | (r << half);
}

// word w of u = x F (non-systematic codes) for the lane's path: the
// transform is an involution, applied here on the lane's scratch column
static __device__ void nonsys_transform(const Ctx &c, int cl)
{
    const int NW = c.N >= 32 ? c.N >> 5 : 1;
    uint32_t *ns = (uint32_t *)(c.gm + c.P->lay.ns_off);
    const uint32_t cap = c.P->lay.ns_words;
    for (int w = 0; w < NW; ++w) st(c, ns, w * 32 + c.lane, cap, xhat_word(c, w, c.lane, cl), 512u);
    // strides >= 32 positions: whole words
    for (int sw = NW >> 1; sw >= 1; sw >>= 1)
        for (int w = 0; w < NW; ++w)
            if ((w & sw) == 0) {
                uint32_t a = ld(c, ns, w * 32 + c.lane, cap, 512u) ^ ld(c, ns, (w + sw) * 32 + c.lane, cap, 512u);
                st(c, ns, w * 32 + c.lane, cap, a, 512u);
            }
    // strides < 32 inside each word: x_i ^= x_{i+s} for i with bit s clear
    const int top = c.N < 32 ? c.N : 32;
    for (int w = 0; w < NW; ++w) {
        uint32_t v = ld(c, ns, w * 32 + c.lane, cap, 512u);
        const uint32_t lo[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
#pragma unroll
        for (int k = 0; k < 5; ++k)
            if ((1 << k) < top) v ^= (v >> (1 << k)) & lo[k];
        st(c, ns, w * 32 + c.lane, cap, v, 512u);
    }
}

__device__ __forceinline__ uint32_t uword(const Ctx &c, int w, int col, int cl)
{
    if (c.P->code.systematic) return xhat_word(c, w, col, cl);
    const uint32_t *ns = (const uint32_t *)(c.gm + c.P->lay.ns_off);
    return ld(c, ns, w * 32 + col, c.P->lay.ns_words, 512u);
}

// CRC check of the lane's path (Sec. IV-B): the first K_info bits of u_A feed
// the CRC register (MSB first, starting at 0), the last c are compared with
// the remainder.  The comparison is linear in the codeword, so it is computed
// as a syndrome: one table lookup per codeword byte (XOR of the columns of the
// byte's one-bits), zero when the check passes.
static __device__ bool crc_check(const Ctx &c, int cl)
{
    const DevCode &cd = c.P->code;
    if (cd.crc_len == 0) return true;
    const int NB = c.N >> 3;
    uint32_t s = 0;
    for (int w0 = 0; w0 * 4 < NB; w0 += 4) {
        uint32_t x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = (w0 + u) * 4 < NB ? uword(c, w0 + u, c.lane, cl) : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = (w0 + u) * 4 + j;
                if (q < NB) s ^= __ldg(&cd.syn[(q << 8) | ((x[u] >> (8 * j)) & 0xFFu)]);
            }
    }
    return s == 0;
}

// ---------------------------------------------------------------------------
// Decode the frames of one task: list positions [pos0, pos0 + 32/L).
template <class Qt, bool NODES>
__device__ void decode_task(Ctx &c, int pos0, int count)
{
    typedef typename Qt::V V;
    PSCL_PROF_T0(t_load);
    const Item &P = *c.P;
    const DevCode &cd = P.code;
    int32_t *fids = (int32_t *)(c.sm + P.lay.src_off) + P.lay.info_words;  // 32 frame ids
    // frame id of this lane's frame (-1: none)
    const int pos = pos0 + c.fiw;
    {
        int frame = -1;
        if (pos < count) frame = P.frame_list ? __ldg(&P.frame_list[pos]) : pos;
        if (c.slot == 0) fids[c.fiw] = frame;
    }
    __syncwarp();
    // layer 0: channel LLRs of the warp's frames, quantised and packed
    {
        uint32_t *l0 = llr_layer(c, 0);
        const uint32_t cap = P.lay.llr_words[0];
        const int rows = (c.N + Qt::EPW - 1) / Qt::EPW;
        const int stride = c.N - cd.P;
        const bool vec = cd.P == 0 && c.N % (4 * Qt::EPW) == 0 && (reinterpret_cast<uintptr_t>(P.llr) & 15u) == 0;
        if (vec) {
            // nothing punctured: lane l takes quads of frame l mod (32/L), reads
            // a quad's 4 x EPW LLRs with 16-byte loads (two quads in flight)
            // and writes it with one 16-byte store
            const int totalq = (rows >> 2) * c.fpw;
            for (int w0 = c.lane; w0 < totalq; w0 += 64) {
                float v[2][4 * Qt::EPW];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int wi = w0 + 32 * u;
                    const int q = wi / c.fpw, fr = wi - q * c.fpw;
                    const int f = wi < totalq ? fids[fr] : -1;
#pragma unroll
                    for (int e = 0; e < Qt::EPW; ++e) {
                        float4 x = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
                        if (f >= 0) {
                            const float4 *a = reinterpret_cast<const float4 *>(
                                &P.llr[(size_t)f * (size_t)stride + (size_t)(q * 4 * Qt::EPW + 4 * e)]);
                            x = P.llr_cg ? __ldcg(a) : __ldg(a);
                        }
                        v[u][4 * e] = x.x;
                        v[u][4 * e + 1] = x.y;
                        v[u][4 * e + 2] = x.z;
                        v[u][4 * e + 3] = x.w;
                    }
                }
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const int wi = w0 + 32 * u;
                    if (wi < totalq) {
                        const int q = wi / c.fpw, fr = wi - q * c.fpw;
                        uint32_t w[4];
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            w[k] = 0u;
#pragma unroll
                            for (int e = 0; e < Qt::EPW; ++e) {
                                const uint32_t qv = Qt::quant(v[u][k * Qt::EPW + e]);
                                w[k] |= Qt::EPW == 1 ? qv : (qv << (e * Qt::BITS));
                            }
                        }
                        const int idx = qa(4 * q, fr, c.fpw);
                        if (PSCL_OK_IDX(c, idx + 3, cap, 1024u))
                            *reinterpret_cast<uint4 *>(l0 + idx) = make_uint4(w[0], w[1], w[2], w[3]);
                    }
                }
            }
        } else {
            // punctured codes: lane l takes frame l mod (32/L) (its rows in turn,
            // the positions through the code's input index): each lane has eight
            // loads in flight before it quantises and stores
            constexpr int U = 8 / Qt::EPW;
            const int total = rows * c.fpw;
            for (int w0 = c.lane; w0 < total; w0 += 32 * U) {
                float x[U][Qt::EPW];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int wi = w0 + 32 * u;
                    const int row = wi / c.fpw, fr = wi - row * c.fpw;
                    const int f = wi < total ? fids[fr] : -1;
#pragma unroll
                    for (int e = 0; e < Qt::EPW; ++e) {
                        const int i = row * Qt::EPW + e;
                        x[u][e] = 0.0f;
                        if (f >= 0 && i < c.N) {
                            const int col = __ldg(&cd.in_index[i]);
                            if (col >= 0) {
                                const float *a = &P.llr[(size_t)f * (size_t)stride + col];
                                x[u][e] = P.llr_cg ? __ldcg(a) : __ldg(a);
                            }
                        }
                    }
                }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int wi = w0 + 32 * u;
                    if (wi < total) {
                        const int row = wi / c.fpw, fr = wi - row * c.fpw;
                        uint32_t word = 0;
#pragma unroll
                        for (int e = 0; e < Qt::EPW; ++e) {
                            const uint32_t q = Qt::quant(x[u][e]);
                            word |= Qt::EPW == 1 ? q : (q << (e * Qt::BITS));
                        }
                        st(c, l0, qa(row, fr, c.fpw), cap, word, 1024u);
                    }
                }
            }
        }
    }
    __syncwarp();
    c.n_active = 1;
    tab_fill(c.idxL, c.slot);
    tab_fill(c.idxS, c.slot);
    V pm = Qt::zero();
    PSCL_PROF_ADD(12, t_load);
    // walk the node schedule
    for (int i = 0; i < c.n_ops; ++i) {
        const uint32_t op = __ldg(&c.ops[i]);
        const int d = op_depth(op);
        PSCL_PROF_T0(t_op);
        switch (op_code(op)) {
        case OP_F: op_f<Qt>(c, d); break;
        case OP_G: op_g<Qt>(c, d); break;
        case OP_COMB: op_comb(c, d, op_side(op)); break;
        case OP_RSUB: {
            const uint32_t fz = op >> 16;
            switch (c.N >> d) {
            case 2: op_rsub<Qt, 2, NODES>(c, d, op_side(op), fz, pm); break;
            case 4: op_rsub<Qt, 4, NODES>(c, d, op_side(op), fz, pm); break;
            case 8: op_rsub<Qt, 8, NODES>(c, d, op_side(op), fz, pm); break;
            default: op_rsub<Qt, 8, NODES>(c, d, op_side(op), fz, pm); break;  // host emits S <= 8
            }
            break;
        }
        case OP_RSUB4: {
            const uint32_t fz = op >> 16;
            // the host emits 16-leaf quads for float schedules only
            if constexpr (!Qt::FIXED) op_rsub4<Qt, 4, NODES>(c, d, op_side(op), op_t(op), fz, pm);
            break;
        }
        case OP_RSUB2: {
            const uint32_t fz = op >> 16;
            switch (c.N >> d) {
            case 4: op_rsub2<Qt, 2, NODES>(c, d, op_side(op), op_t(op), fz, pm); break;
            case 8: op_rsub2<Qt, 4, NODES>(c, d, op_side(op), op_t(op), fz, pm); break;
            default: op_rsub2<Qt, 8, NODES>(c, d, op_side(op), op_t(op), fz, pm); break;  // host emits 2H <= 16
            }
            break;
        }
        default:
            if constexpr (NODES) op_node<Qt>(c, d, (int)op_type(op), op_side(op), op_t(op), pm);
            break;
        }
        __syncwarp();
        PSCL_PROF_ADD(op_code(op) == OP_NODE ? 7 + (int)op_type(op) : (int)op_code(op), t_op);
    }
    PSCL_PROF_T0(t_fin);
    // final selection (Sec. IV-B): best metric among paths passing the CRC
    const int cl = c.seg + tab_get(c.idxS, 1);
    if (!cd.systematic) {
        nonsys_transform(c, cl);
        __syncwarp();
    }
    const bool active = c.slot < c.n_active;
    const bool ok = active && crc_check(c, cl);
    uint64_t key = active ? (((uint64_t)(ok ? 0u : 1u) << 40) | ((uint64_t)Qt::key(pm) << 8) | (uint64_t)c.slot)
                          : ~0ull;
    for (int m = 1; m < c.L; m <<= 1) {
        uint64_t o = shfl64_xor(key, m);
        key = o < key ? o : key;
    }
    const int win = (int)(key & 0xFFu);
    const bool wok = ((key >> 40) & 1u) == 0;
    const int wcol = c.seg + win;
    const int wcl = __shfl_sync(PSCL_FULL, cl, wcol);
    // frame ids from shared memory (not kept in registers across the walk)
    const int32_t *fid = (const int32_t *)(c.sm + P.lay.src_off) + P.lay.info_words;
    const int frame = fid[c.fiw];
    if (frame >= 0) {
        if (c.slot == 0) {
            bool pass = wok;
            if (!pass && P.next_list) {
                const int at = atomicAdd(P.next_count, 1);
                P.next_list[at] = frame;
            }
            P.status_out[frame] = (pass ? 1 : 0) | (P.stage_L << 8) | (win << 16);
        }
        if (P.pm_out) {
            for (int s = c.slot; s < P.L_out; s += c.L)
                P.pm_out[(size_t)frame * (size_t)P.L_out + s] = (s == c.slot && active) ? Qt::to_float(pm)
                                                                                        : __uint_as_float(0x7F800000u);
        }
    }
    // info bits of each frame's winning path, the whole warp on one frame at
    // a time: a lane takes four codeword bytes per step, looks up their info
    // bits (table per byte) and ORs them into a bit buffer in shared memory
    // (u_A order, LSB first in 32-bit words); then the lanes write the bytes
    // out MSB first.
    const int nbytes = (cd.kinfo + 7) >> 3;
    const int NB = c.N >> 3;
    uint32_t *buf = (uint32_t *)(c.sm + P.lay.src_off);  // info_words words: K_info bits
    for (int f = 0; f < c.fpw; ++f) {
        const int fr = fid[f];
        const int wc = __shfl_sync(PSCL_FULL, wcol, f * c.L);
        const int wl = __shfl_sync(PSCL_FULL, wcl, f * c.L);
        if (fr < 0) continue;  // warp-uniform
        __syncwarp();
        for (int w = c.lane; w < (int)P.lay.info_words; w += 32) buf[w] = 0u;
        __syncwarp();
        for (int q0 = 4 * c.lane; q0 < NB; q0 += 128) {
            const uint32_t x = uword(c, q0 >> 2, wc, wl);
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int q = q0 + j;
                if (q < NB) {
                    const int k = __ldg(&cd.ext_pos[q]);
                    const int cnt = __ldg(&cd.ext_pos[q + 1]) - k;
                    if (cnt > 0) {
                        const uint32_t v = __ldg(&cd.ext[(q << 8) | ((x >> (8 * j)) & 0xFFu)]);
                        atomicOr(&buf[k >> 5], v << (k & 31));
                        if ((k & 31) + cnt > 32) atomicOr(&buf[(k >> 5) + 1], v >> (32 - (k & 31)));
                    }
                }
            }
        }
        __syncwarp();
        for (int b = c.lane; b < nbytes; b += 32) {
            const uint32_t byte = (buf[b >> 2] >> (8 * (b & 3))) & 0xFFu;
            P.info_out[(size_t)fr * (size_t)nbytes + b] = (uint8_t)(__brev(byte) >> 24);
        }
    }
    __syncwarp();
    PSCL_PROF_ADD(13, t_fin);
}

// copy an item into the warp's shared slice and set the lane roles
__device__ __forceinline__ void load_item(Ctx &c, const Item *src, const KParams &K, bool batch)
{
    uint32_t *dst = (uint32_t *)c.sm;
    const uint32_t *from = (const uint32_t *)src;
    __syncwarp();
    for (int i = c.lane; i < (int)(sizeof(Item) / 4); i += 32) dst[i] = from[i];
    __syncwarp();
    if (batch && c.lane == 0) {
        Item *it = (Item *)c.sm;
        it->llr = K.llr_pool + it->llr_off;
        it->info_out = K.info_pool + it->info_off;
        it->status_out = K.status_pool + it->status_off;
        it->pm_out = nullptr;
    }
    __syncwarp();
    const Item &it = *c.P;
    if (c.lane < 3 * kMaxLayers) {
        // lanes 0..11 LLR layers, 12..23 BL, 24..31 BR (and 32..35 below)
        const int kind = c.lane / kMaxLayers, d = c.lane - kind * kMaxLayers;
        const uint32_t mask = kind == 0 ? it.lay.llr_smem : (kind == 1 ? it.lay.bl_smem : it.lay.br_smem);
        const uint32_t off = kind == 0 ? it.lay.llr_off[d] : (kind == 1 ? it.lay.bl_off[d] : it.lay.br_off[d]);
        ptab(c)[c.lane] = (uint32_t *)((((mask >> d) & 1u) ? c.sm : c.gm) + off);
    }
    if (c.lane < 3 * kMaxLayers - 32) {
        const int d = 32 - 2 * kMaxLayers + c.lane;
        ptab(c)[32 + c.lane] = (uint32_t *)((((it.lay.br_smem >> d) & 1u) ? c.sm : c.gm) + it.lay.br_off[d]);
    }
    __syncwarp();
    c.ops = it.ops;
    c.n_ops = it.n_ops;
    c.L = it.L;
    c.fpw = 32 / it.L;
    c.slot = c.lane & (it.L - 1);
    c.seg = c.lane - c.slot;
    c.fiw = c.lane / it.L;
    c.N = it.code.N;
    c.n = it.code.n;
    c.n_active = 1;
}

// Persistent kernel: each warp decodes task after task.  With a task list
// (uneven batches) the next task comes from a device counter, so warps that
// drew short frames take more of them; otherwise warps stride over the
// frames of the single item.
// The registers are capped as for MINB blocks of four warps per SM: the
// node-capable variant as for 4 (128 registers), the node-free one as for 5
// (96) or 7 (72).  The cap does not fix the block size: blocks of 1, 2, 4
// or 8 warps (frames per block, a tuned knob) all fit it.
template <class Qt, bool NODES, int MINB>
__global__ void __maxnreg__((65536 / (128 * MINB)) & ~7) scl_kernel(const __grid_constant__ KParams K)
{
    extern __shared__ __align__(16) char smem[];
    Ctx c;
    const int warp = threadIdx.x >> 5;
    c.lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    c.sm = smem + (size_t)warp * K.smem_per_warp;
    c.gm = K.gmem + (size_t)gwarp * K.gmem_per_warp;
    c.P = (const Item *)c.sm;
#ifdef PSCL_OPPROF
    c.prof = K.op_cycles;
#endif
    if (K.tasks == nullptr) {
        load_item(c, &K.single, K, false);
        const Item &it = *c.P;
        const int count = it.frame_list ? *it.list_count : it.n_frames;
        const int n_tasks = (count + c.fpw - 1) / c.fpw;
        for (int task = gwarp; task < n_tasks; task += K.total_warps) decode_task<Qt, NODES>(c, task * c.fpw, count);
        return;
    }
    int cur = -1;
    for (;;) {
        int t = 0;
        if (c.lane == 0) t = atomicAdd(K.task_ctr, 1);
        t = __shfl_sync(PSCL_FULL, t, 0);
        if (t >= K.n_tasks) break;
        const int2 tk = K.tasks[t];
        if (tk.x != cur) {
            load_item(c, K.items + tk.x, K, true);
            cur = tk.x;
        }
        decode_task<Qt, NODES>(c, tk.y, c.P->n_frames);
    }
}

}  // namespace pscl
