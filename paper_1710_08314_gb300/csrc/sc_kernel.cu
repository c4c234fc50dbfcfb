// sc_kernel.cu -- successive-cancellation decoding (the list of one, Sec.
// II-B), one warp per frame, for the SC algorithm and the first stage of the
// adaptive schedules (FA, PA).
//
// With a single path there is nothing to select: at every information leaf or
// pruned node the least-penalty candidate wins, which is the hard decision
// (R1, and an information leaf), the cheaper of the two words (REP), the hard
// decision with the least reliable position flipped when its parity is odd
// (SPC), or the zero word (R0, frozen leaf); the path metric adds the
// winner's penalty (float) or stays 0 (fixed point: it is normalised after
// every step, and a list of one has its own metric as the minimum).  So the
// warp spends its lanes on the elements of a node instead of on paths:
//   - LLR layers 1..n of the frame live in the warp's shared-memory slice
//     (layer d holds the N/2^d LLRs of the current depth-d node); layer 0 is
//     read from the channel LLRs in global memory (quantised on the fly);
//   - the partial sums are one N-bit array (node at leaf offset o of size S
//     owns bits o..o+S-1; the h step XORs the right half into the left);
//   - f and g run over a node's words with the lanes side by side; node
//     penalties are sums over the node's positions in a balanced pairwise
//     tree over index order (per-lane chunks, then a butterfly across lanes),
//     the same tree the list decoder and the oracle use.
// The schedule is the pruned tree of the list decoder, each step carrying its
// node's leaf offset (bits 16..31); subtrees of up to 16 leaves are one step,
// decoded in registers by every lane alike together with the pruned nodes
// inside them, and so are the node handlers of nodes up to 8 positions.  The warp reads its schedule 32 steps
// at a time (a lane per step) and passes the steps round by shuffles.
#include <map>
#include <mutex>

#include "scl_kernel.cuh"

namespace pscl {

template <class Qt>
struct ScFrame {
    typedef typename Qt::V V;
    const Item &P;
    char *sm;
    int lane, N;
    const float *llr;
    uint32_t *sb;  // partial-sum bits

    __device__ ScFrame(const Item &p, char *s, int l, int frame)
        : P(p), sm(s), lane(l), N(p.code.N)
    {
        llr = P.llr + (size_t)frame * (size_t)(N - P.code.P);
        sb = (uint32_t *)(sm + P.lay.bl_off[0]);
    }
    __device__ uint32_t *layer(int d) const { return (uint32_t *)(sm + P.lay.llr_off[d]); }

    // word w of layer 0: channel LLRs of positions w*EPW.., quantised
    __device__ uint32_t word0(int w) const
    {
        uint32_t word = 0;
#pragma unroll
        for (int e = 0; e < Qt::EPW; ++e) {
            const int i = w * Qt::EPW + e;
            float x = 0.0f;
            if (i < N) {
                const int col = P.code.P ? __ldg(&P.code.in_index[i]) : i;
                if (col >= 0) x = P.llr_cg ? __ldcg(&llr[col]) : __ldg(&llr[col]);
            }
            const uint32_t q = Qt::quant(x);
            word |= Qt::EPW == 1 ? q : (q << (e * Qt::BITS));
        }
        return word;
    }
    __device__ uint32_t word(int d, int w) const { return d == 0 ? word0(w) : layer(d)[w]; }
    __device__ V elem(int d, int i) const { return Qt::elem(word(d, i / Qt::EPW), i % Qt::EPW); }

    // bits o..o+k-1 of the partial sums (k <= 32, not crossing a word)
    __device__ uint32_t bits(int o, int k) const
    {
        const uint32_t w = sb[o >> 5] >> (o & 31);
        return k >= 32 ? w : (w & ((1u << k) - 1u));
    }

    // layer d+1 = f (left child) or g (right child, partial sums of the
    // left child at leaf offset o) of the depth-d node
    template <bool G>
    __device__ void fg(int d, int o)
    {
        constexpr uint32_t M1 = (1u << Qt::EPW) - 1u;
        const int S = N >> d, H = S >> 1;
        uint32_t *out = layer(d + 1);
        if (H >= Qt::EPW) {
            const int HW = H / Qt::EPW;
            if (d > 0 && HW >= 128) {
                // quads of words: 16-byte accesses
                const uint4 *in4 = (const uint4 *)layer(d);
                uint4 *out4 = (uint4 *)out;
                const int HQ = HW >> 2;
                for (int q = lane; q < HQ; q += 32) {
                    const uint4 a = in4[q], b = in4[q + HQ];
                    uint4 r;
                    if (G) {
                        const uint32_t s = bits(o + 4 * q * Qt::EPW, 4 * Qt::EPW);
                        r = make_uint4(Qt::G(a.x, b.x, s & M1), Qt::G(a.y, b.y, (s >> Qt::EPW) & M1),
                                       Qt::G(a.z, b.z, (s >> (2 * Qt::EPW)) & M1),
                                       Qt::G(a.w, b.w, (s >> (3 * Qt::EPW)) & M1));
                    } else {
                        r = make_uint4(Qt::F(a.x, b.x), Qt::F(a.y, b.y), Qt::F(a.z, b.z), Qt::F(a.w, b.w));
                    }
                    out4[q] = r;
                }
            } else {
                for (int w = lane; w < HW; w += 32) {
                    const uint32_t a = word(d, w), b = word(d, w + HW);
                    out[w] = G ? Qt::G(a, b, bits(o + w * Qt::EPW, Qt::EPW)) : Qt::F(a, b);
                }
            }
        } else if (lane == 0) {
            // the node fits in one word: its halves are sub-words of it
            const uint32_t wd = word(d, 0);
            out[0] = G ? Qt::G(wd, wd >> (H * Qt::BITS), bits(o, H)) : Qt::F(wd, wd >> (H * Qt::BITS));
        }
    }

    // h step of the node at leaf offset o whose children have Hc leaves
    __device__ void comb(int Hc, int o)
    {
        if (Hc >= 32) {
            const int W = Hc >> 5, base = o >> 5;
            for (int w = lane; w < W; w += 32) sb[base + w] ^= sb[base + W + w];
        } else if (lane == 0) {
            const uint32_t m = (1u << Hc) - 1u, sh = (uint32_t)(o & 31);
            const uint32_t wd = sb[o >> 5];
            sb[o >> 5] = wd ^ (((wd >> (sh + Hc)) & m) << sh);
        }
    }

    // write bits o..o+S-1 of the partial sums: S >= 32 from per-row words
    // (row r: bits 32r..32r+31 of the node), S < 32 into one word
    __device__ void put_small(int o, int S, uint32_t v)
    {
        if (lane == 0) {
            const uint32_t m = S >= 32 ? 0xFFFFFFFFu : ((1u << S) - 1u), sh = (uint32_t)(o & 31);
            sb[o >> 5] = (sb[o >> 5] & ~(m << sh)) | ((v & m) << sh);
        }
    }

    // sum over the node's positions (balanced pairwise tree over index order)
    // of pen(value); all lanes get the sum.  Lane L takes the C = S/32
    // consecutive positions L*C.. (S >= 32) or position L (S < 32).
    template <class Pen>
    __device__ V tree_sum(int d, int S, const Pen &pen) const
    {
        V v = Qt::zero();
        if (S >= 32) {
            const int C = S >> 5;
            TreeSum<Qt> t;
            for (int k = 0; k < C; ++k) v = t.push(pen(elem(d, lane * C + k)), k);
        } else if (lane < S) {
            v = pen(elem(d, lane));
        }
        // lanes 2k and 2k+1 hold neighbouring runs: pairwise up the tree
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) {
            const V o = (V)__shfl_xor_sync(PSCL_FULL, v, m);
            v = (lane & m) ? Qt::add(o, v) : Qt::add(v, o);
        }
        return v;
    }

    // hard decisions of the node into the partial sums; returns their parity
    __device__ int hard(int d, int o, int S)
    {
        int par = 0;
        if (S >= 32) {
            for (int r = 0; r < (S >> 5); ++r) {
                const uint32_t b = __ballot_sync(PSCL_FULL, elem(d, 32 * r + lane) < 0);
                par ^= __popc(b) & 1;
                if (lane == 0) sb[(o >> 5) + r] = b;
            }
        } else {
            const uint32_t b = __ballot_sync(PSCL_FULL, lane < S && elem(d, lane < S ? lane : 0) < 0);
            par = __popc(b) & 1;
            put_small(o, S, b);
        }
        return par;
    }

    __device__ void fill(int o, int S, uint32_t v)
    {
        if (S >= 32) {
            for (int w = lane; w < (S >> 5); w += 32) sb[(o >> 5) + w] = v;
        } else {
            put_small(o, S, v);
        }
    }

    // the S (<= 8) values of a depth-d node, read by every lane (one shared
    // load serves the whole warp)
    template <int S>
    __device__ void load_small(int d, V (&a)[S]) const
    {
        constexpr int NW = (S + Qt::EPW - 1) / Qt::EPW;
        if (d == 0) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t wd = word0(w);
#pragma unroll
                for (int e = 0; e < Qt::EPW; ++e)
                    if (w * Qt::EPW + e < S) a[w * Qt::EPW + e] = Qt::elem(wd, e);
            }
        } else {
            const uint32_t *in = layer(d);
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t wd = in[w];
#pragma unroll
                for (int e = 0; e < Qt::EPW; ++e)
                    if (w * Qt::EPW + e < S) a[w * Qt::EPW + e] = Qt::elem(wd, e);
            }
        }
    }

    // a node of S <= 16 positions whose values every lane holds: every lane
    // takes the same decision, so no lane has to wait for another; returns
    // the node's partial-sum bits
    template <int S>
    __device__ uint32_t node_regs(const V (&a)[S], int type, V &pm) const
    {
        uint32_t h = 0;
#pragma unroll
        for (int i = 0; i < S; ++i) h |= (uint32_t)(a[i] < 0) << i;
        if (type == NT_R1) return h;
        if (type == NT_R0) {
            if (!Qt::FIXED) {
                TreeSum<Qt> t0;
                V p0 = Qt::zero();
#pragma unroll
                for (int i = 0; i < S; ++i) p0 = t0.push(a[i] < 0 ? Qt::absv(a[i]) : Qt::zero(), i);
                pm = Qt::add(pm, p0);
            }
            return 0u;
        }
        if (type == NT_REP) {
            TreeSum<Qt> t0, t1;
            V p0 = Qt::zero(), p1 = Qt::zero();
#pragma unroll
            for (int i = 0; i < S; ++i) {
                p0 = t0.push(a[i] < 0 ? Qt::absv(a[i]) : Qt::zero(), i);
                p1 = t1.push(a[i] > 0 ? Qt::absv(a[i]) : Qt::zero(), i);
            }
            const V c0 = Qt::add(Qt::FIXED ? Qt::zero() : pm, p0), c1 = Qt::add(Qt::FIXED ? Qt::zero() : pm, p1);
            const bool ones = Qt::key(c1) < Qt::key(c0);
            if (!Qt::FIXED) pm = ones ? c1 : c0;
            return ones ? 0xFFFFFFFFu : 0u;
        }
        // SPC: odd parity flips the least reliable position (smallest (|a|, i))
        if (__popc(h) & 1) {
            int r0 = 0;
            uint32_t kb = Qt::key(Qt::absv(a[0]));
#pragma unroll
            for (int i = 1; i < S; ++i) {
                const uint32_t k = Qt::key(Qt::absv(a[i]));
                if (k < kb) {
                    kb = k;
                    r0 = i;
                }
            }
            h ^= 1u << r0;
            if (!Qt::FIXED) pm = Qt::add(pm, Qt::add(Qt::zero(), Qt::from_key(kb)));
        }
        return h;
    }

    // a node of S <= 8 positions: every lane reads all of them
    template <int S>
    __device__ void node_small(int d, int o, int type, V &pm)
    {
        V a[S];
        load_small<S>(d, a);
        put_small(o, S, node_regs<S>(a, type, pm));
    }

    // a subtree of S leaves (S = 2, 4, 8, 16) decoded in registers by every
    // lane alike: f, g and h of Sec. II-B, information leaves take the hard
    // decision, frozen leaves add their penalty; with NODES, a pruned node
    // inside it (its type in desc: 3 bits per node of the enclosing 16-leaf
    // group, node h of the group in heap order at bits 3(h-1)) is decided as
    // one.  Returns its S bits.
    template <int S, bool NODES>
    __device__ uint32_t rsub(const V (&a)[S], uint32_t fz, V &pm, uint64_t desc, int h) const
    {
        if constexpr (S == 1) {
            if (fz & 1u) {
                if (!Qt::FIXED) pm = Qt::add(pm, a[0] < 0 ? Qt::absv(a[0]) : Qt::zero());
                return 0u;
            }
            return (uint32_t)(a[0] < 0);
        } else {
            if constexpr (NODES) {
                const int type = (int)((desc >> (3 * (h - 1))) & 7u);
                if (type != 0) return node_regs<S>(a, type, pm);
            }
            constexpr int H = S / 2;
            V l[H], r[H];
#pragma unroll
            for (int i = 0; i < H; ++i) l[i] = Qt::f1(a[i], a[i + H]);
            const uint32_t bl = rsub<H, NODES>(l, fz, pm, desc, 2 * h);
#pragma unroll
            for (int i = 0; i < H; ++i) r[i] = Qt::g1(a[i], a[i + H], (bl >> i) & 1u);
            const uint32_t br = rsub<H, NODES>(r, fz >> H, pm, desc, 2 * h + 1);
            constexpr uint32_t m = (1u << H) - 1u;
            return ((bl ^ br) & m) | ((br & m) << H);
        }
    }

    // nodes: the host found pruned nodes inside the subtree (step field t)
    template <int S>
    __device__ void rsub_step(int d, int o, bool nodes, V &pm)
    {
        V a[S];
        load_small<S>(d, a);
        const uint32_t fz = ~(__ldg(&P.code.amask[o >> 5]) >> (o & 31));
        if (nodes) {
            // node types of the 16-leaf groups, after the schedule (8-byte aligned)
            const uint64_t *desc = reinterpret_cast<const uint64_t *>(P.ops + ((P.n_ops + 1) & ~1));
            put_small(o, S, rsub<S, true>(a, fz, pm, __ldg(&desc[o >> 4]), 16 / S + (o & 15) / S));
        } else {
            put_small(o, S, rsub<S, false>(a, fz, pm, 0, 1));
        }
    }

    // a 32-leaf subtree as one step: f into registers, the left 16-leaf
    // subtree, g from the node's values read again, the right one, and the
    // node's h; t bit 0 / bit 1: pruned nodes inside the left / right half
    __device__ void rsub2_step(int d, int o, int t, V &pm)
    {
        constexpr int H = 16;
        const uint32_t fz = ~(__ldg(&P.code.amask[o >> 5]) >> (o & 31));
        const uint64_t *desc = reinterpret_cast<const uint64_t *>(P.ops + ((P.n_ops + 1) & ~1));
        uint32_t bl, br;
        {
            V a[2 * H], l[H];
            load_small<2 * H>(d, a);
#pragma unroll
            for (int i = 0; i < H; ++i) l[i] = Qt::f1(a[i], a[i + H]);
            bl = (t & 1) ? rsub<H, true>(l, fz, pm, __ldg(&desc[o >> 4]), 1) : rsub<H, false>(l, fz, pm, 0, 1);
        }
        {
            V a[2 * H], r[H];
            load_small<2 * H>(d, a);
#pragma unroll
            for (int i = 0; i < H; ++i) r[i] = Qt::g1(a[i], a[i + H], (bl >> i) & 1u);
            br = (t & 2) ? rsub<H, true>(r, fz >> H, pm, __ldg(&desc[(o >> 4) + 1]), 1)
                         : rsub<H, false>(r, fz >> H, pm, 0, 1);
        }
        put_small(o, 2 * H, ((bl ^ br) & 0xFFFFu) | (br << H));
    }

    // a leaf or pruned node at depth d, leaf offset o
    __device__ void node(int d, int o, int type, V &pm)
    {
        const int S = N >> d;
        switch (S) {
        case 1: node_small<1>(d, o, type, pm); return;
        case 2: node_small<2>(d, o, type, pm); return;
        case 4: node_small<4>(d, o, type, pm); return;
        case 8: node_small<8>(d, o, type, pm); return;
        default: break;
        }
        if (type == NT_R0) {
            const V pen = tree_sum(d, S, [](V a) { return a < 0 ? Qt::absv(a) : Qt::zero(); });
            if (!Qt::FIXED) pm = Qt::add(pm, pen);
            fill(o, S, 0u);
        } else if (type == NT_R1) {
            hard(d, o, S);  // the hard decision is the zero-penalty candidate
        } else if (type == NT_REP) {
            const V p0 = tree_sum(d, S, [](V a) { return a < 0 ? Qt::absv(a) : Qt::zero(); });
            const V p1 = tree_sum(d, S, [](V a) { return a > 0 ? Qt::absv(a) : Qt::zero(); });
            const V c0 = Qt::add(Qt::FIXED ? Qt::zero() : pm, p0), c1 = Qt::add(Qt::FIXED ? Qt::zero() : pm, p1);
            const bool ones = Qt::key(c1) < Qt::key(c0);
            if (!Qt::FIXED) pm = ones ? c1 : c0;
            fill(o, S, ones ? 0xFFFFFFFFu : 0u);
        } else {
            // SPC: hard decision; odd parity flips the least reliable position
            const int par = hard(d, o, S);
            if (par) {
                // (|alpha|, index) minimum over the node
                uint64_t best = ~0ull;
                if (S >= 32) {
                    const int C = S >> 5;
                    for (int k = 0; k < C; ++k) {
                        const int i = lane * C + k;
                        const uint64_t key = ((uint64_t)Qt::key(Qt::absv(elem(d, i))) << 32) | (uint32_t)i;
                        best = key < best ? key : best;
                    }
                } else if (lane < S) {
                    best = ((uint64_t)Qt::key(Qt::absv(elem(d, lane))) << 32) | (uint32_t)lane;
                }
#pragma unroll
                for (int m = 1; m < 32; m <<= 1) {
                    const uint64_t x = shfl64_xor(best, m);
                    best = x < best ? x : best;
                }
                const int r0 = (int)(uint32_t)best;
                if (!Qt::FIXED) pm = Qt::add(pm, Qt::add(Qt::zero(), Qt::from_key((uint32_t)(best >> 32))));
                __syncwarp();
                if (lane == 0) sb[(o + r0) >> 5] ^= 1u << ((o + r0) & 31);
            }
        }
    }
};

// codeword word w (positions 32w..32w+31) of the decoded frame: u for
// non-systematic codes (transformed in place), x for systematic ones
template <class Qt>
__device__ void sc_finish(const Item &P, char *sm, int lane, int frame, float pm)
{
    const DevCode &cd = P.code;
    const int N = cd.N, NW = N >= 32 ? N >> 5 : 1;
    uint32_t *sb = (uint32_t *)(sm + P.lay.bl_off[0]);
    if (!cd.systematic) {
        // u = x F (the transform is an involution): word strides, then bits
        for (int sw = NW >> 1; sw >= 1; sw >>= 1) {
            for (int w = lane; w < NW; w += 32)
                if ((w & sw) == 0) sb[w] ^= sb[w + sw];
            __syncwarp();
        }
        const int top = N < 32 ? N : 32;
        const uint32_t lo[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
        for (int w = lane; w < NW; w += 32) {
            uint32_t v = sb[w];
#pragma unroll
            for (int k = 0; k < 5; ++k)
                if ((1 << k) < top) v ^= (v >> (1 << k)) & lo[k];
            sb[w] = v;
        }
        __syncwarp();
    }
    // CRC as a syndrome over the codeword bytes (Sec. IV-B), lanes side by side
    const int NB = N >> 3;
    bool ok = true;
    if (cd.crc_len > 0) {
        uint32_t s = 0;
        for (int q = lane; q < NB; q += 32) s ^= __ldg(&cd.syn[(q << 8) | ((sb[q >> 2] >> (8 * (q & 3))) & 0xFFu)]);
#pragma unroll
        for (int m = 1; m < 32; m <<= 1) s ^= __shfl_xor_sync(PSCL_FULL, s, m);
        ok = s == 0;
    }
    if (lane == 0) {
        if (!ok && P.next_list) {
            const int at = atomicAdd(P.next_count, 1);
            P.next_list[at] = frame;
        }
        P.status_out[frame] = (ok ? 1 : 0) | (P.stage_L << 8);
    }
    if (P.pm_out)
        for (int s = lane; s < P.L_out; s += 32)
            P.pm_out[(size_t)frame * (size_t)P.L_out + s] = s == 0 ? pm : __uint_as_float(0x7F800000u);
    // info bits: per codeword byte, its info bits from a table, ORed into a
    // bit buffer (u_A order, LSB first), then written out MSB first
    uint32_t *buf = (uint32_t *)(sm + P.lay.src_off);
    for (int w = lane; w < (int)P.lay.info_words; w += 32) buf[w] = 0u;
    __syncwarp();
    for (int q = lane; q < NB; q += 32) {
        const int k = __ldg(&cd.ext_pos[q]);
        const int cnt = __ldg(&cd.ext_pos[q + 1]) - k;
        if (cnt > 0) {
            const uint32_t v = __ldg(&cd.ext[(q << 8) | ((sb[q >> 2] >> (8 * (q & 3))) & 0xFFu)]);
            atomicOr(&buf[k >> 5], v << (k & 31));
            if ((k & 31) + cnt > 32) atomicOr(&buf[(k >> 5) + 1], v >> (32 - (k & 31)));
        }
    }
    __syncwarp();
    const int nbytes = (cd.kinfo + 7) >> 3;
    for (int b = lane; b < nbytes; b += 32) {
        const uint32_t byte = (buf[b >> 2] >> (8 * (b & 3))) & 0xFFu;
        P.info_out[(size_t)frame * (size_t)nbytes + b] = (uint8_t)(__brev(byte) >> 24);
    }
    __syncwarp();
}

// resident blocks of four warps per SM the registers are sized for: the
// float slices (N = 2048: 8.7 KB) let six blocks share an SM, the packed
// fixed-point ones more
template <class Qt>
struct ScBlocks {
    static constexpr int value = Qt::EPW == 1 ? 6 : 8;
};

template <class Qt>
__global__ void __launch_bounds__(128, ScBlocks<Qt>::value) sc_kernel(const __grid_constant__ KParams K)
{
    extern __shared__ __align__(16) char smem[];
    typedef typename Qt::V V;
    const Item &P = K.single;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    char *sm = smem + (size_t)warp * K.smem_per_warp;
    const int count = P.frame_list ? *P.list_count : P.n_frames;
    const int N = P.code.N;
    for (int pos = gwarp; pos < count; pos += K.total_warps) {
        const int frame = P.frame_list ? __ldg(&P.frame_list[pos]) : pos;
        ScFrame<Qt> f(P, sm, lane, frame);
        V pm = Qt::zero();
        uint32_t batch = 0;  // 32 schedule steps, one per lane, passed round by shuffles
        for (int i = 0; i < P.n_ops; ++i) {
            if ((i & 31) == 0) batch = i + lane < P.n_ops ? __ldg(&P.ops[i + lane]) : 0u;
            const uint32_t op = __shfl_sync(PSCL_FULL, batch, i & 31);
            const int d = op_depth(op), o = (int)(op >> 16);
            switch (op_code(op)) {
            case OP_F: f.template fg<false>(d, o); break;
            case OP_G: f.template fg<true>(d, o); break;
            case OP_COMB: f.comb(N >> d, o); break;
            case OP_RSUB:
                switch (N >> d) {
                case 2: f.template rsub_step<2>(d, o, op_t(op) != 0, pm); break;
                case 4: f.template rsub_step<4>(d, o, op_t(op) != 0, pm); break;
                case 8: f.template rsub_step<8>(d, o, op_t(op) != 0, pm); break;
                default: f.template rsub_step<16>(d, o, op_t(op) != 0, pm); break;  // the host emits 2, 4, 8 or 16
                }
                break;
            case OP_RSUB2: f.rsub2_step(d, o, op_t(op), pm); break;  // 32 leaves
            default: f.node(d, o, (int)op_type(op), pm); break;
            }
            __syncwarp();
        }
        if (!P.root_special) {
            f.comb(N >> 1, 0);
            __syncwarp();
        }
        sc_finish<Qt>(P, sm, lane, frame, Qt::to_float(pm));
    }
}

static std::mutex g_sc_mu;
static std::map<int, int> g_sc_attr;

template <class Qt>
static cudaError_t sc_set_attr()
{
    int dev, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_sc_mu);
    const int key = dev * 4 + Qt::EPW;
    if (g_sc_attr[key]) return cudaSuccess;
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(sc_kernel<Qt>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) g_sc_attr[key] = 1;
    return e;
}

template <class Qt>
static cudaError_t sc_launch_q(const KParams &p, int grid, int block, size_t smem, cudaStream_t s)
{
    cudaError_t e = sc_set_attr<Qt>();
    if (e != cudaSuccess) return e;
    sc_kernel<Qt><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <class Qt>
static cudaError_t sc_attrs_q(size_t smem, int block, int *bps)
{
    cudaError_t e = sc_set_attr<Qt>();
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, sc_kernel<Qt>, block, smem);
}

cudaError_t launch_sc(int quant, const KParams &p, int grid, int block, size_t smem, cudaStream_t s)
{
    if (quant == 0) return sc_launch_q<QF32>(p, grid, block, smem, s);
    if (quant == 1) return sc_launch_q<QI16>(p, grid, block, smem, s);
    return sc_launch_q<QI8>(p, grid, block, smem, s);
}

cudaError_t sc_attrs(int quant, size_t smem, int block, int *bps)
{
    if (quant == 0) return sc_attrs_q<QF32>(smem, block, bps);
    if (quant == 1) return sc_attrs_q<QI16>(smem, block, bps);
    return sc_attrs_q<QI8>(smem, block, bps);
}

}  // namespace pscl
