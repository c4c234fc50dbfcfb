// api.cu -- host side of libpolarscl: the C ABI declared in include/polarscl.h.
//
// Code descriptors (Sec. III-A genericity: N, frozen set, CRC and puncturing
// are run-time data), the node schedule built per pruning setting (Sec. II-B,
// III-B-2), the per-warp memory layout, the workspace and the launches.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <time.h>

#include <algorithm>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/polarscl.h"
#include "internal.h"

using namespace pscl;

// ---------------------------------------------------------------------------
// errors
static thread_local std::string g_err;

static int fail(int code, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? PSCL_ENOMEM : PSCL_ECUDA, "%s: %s", \
                        #call, cudaGetErrorString(e_));                                       \
    } while (0)

extern "C" const char *pscl_last_error(void) { return g_err.c_str(); }
extern "C" const char *pscl_version(void) { return "polarscl 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// device properties
struct DevProps {
    int sms = 0;
    int smem_optin = 0;
    int smem_per_sm = 0;
    int smem_reserved = 0;  // per block, taken by the runtime
};
static std::mutex g_mu;
static std::map<int, DevProps> g_props;

static int get_props(DevProps *out)
{
    int dev;
    CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_props.find(dev);
    if (it == g_props.end()) {
        DevProps p;
        CU(cudaDeviceGetAttribute(&p.sms, cudaDevAttrMultiProcessorCount, dev));
        CU(cudaDeviceGetAttribute(&p.smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
        CU(cudaDeviceGetAttribute(&p.smem_per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev));
        CU(cudaDeviceGetAttribute(&p.smem_reserved, cudaDevAttrReservedSharedMemoryPerBlock, dev));
        it = g_props.emplace(dev, p).first;
    }
    *out = it->second;
    return PSCL_OK;
}

// ---------------------------------------------------------------------------
// Releasing device memory.  cudaFree (and cudaFreeHost) wait for every kernel
// on the device, and a serving loop's kernel runs until it is stopped or its
// idle budget runs out: a free issued while a server runs on the device would
// stall the caller for that long.  While any server runs on a device, the
// library's own frees on that device are therefore queued and carried out
// when the last server there stops.
static std::mutex g_free_mu;
static std::map<int, int> g_servers_running;                       // per device
static std::map<int, std::vector<std::pair<void *, bool>>> g_deferred;  // (pointer, host)

static void lib_free(void *p, bool host = false)
{
    if (!p) return;
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_free_mu);
        if (g_servers_running[dev] > 0) {
            g_deferred[dev].push_back(std::make_pair(p, host));
            return;
        }
    }
    if (host) cudaFreeHost(p);
    else cudaFree(p);
}

static void server_started(int dev)
{
    std::lock_guard<std::mutex> lk(g_free_mu);
    g_servers_running[dev]++;
}

// the server on `dev` has stopped: release what was queued once none is left
static void server_stopped(int dev)
{
    std::vector<std::pair<void *, bool>> todo;
    {
        std::lock_guard<std::mutex> lk(g_free_mu);
        if (--g_servers_running[dev] > 0) return;
        todo.swap(g_deferred[dev]);
    }
    for (auto &pr : todo) {
        if (pr.second) cudaFreeHost(pr.first);
        else cudaFree(pr.first);
    }
}

// ---------------------------------------------------------------------------
// code descriptor
struct Program {
    uint32_t *d_ops = nullptr;
    int has_nodes = 0;   // contains pruned-node steps
    int n_ops = 0;
    int max_depth = 0;
    int root_special = 0;
};

// measured tuning of one (list size, number format, pruning) of a code
struct Tuning {
    int warps_per_sm = 0;     // warps per SM the shared-memory slices are sized for
    int fuse = 0;             // largest register subtree (leaves)
    int warps_per_block = 0;  // warps of a block (frames per block = warps x 32/L)
    int resident_warps = 0;   // occupancy target selecting the register cap (0 = warps_per_sm)
};

struct pscl_code_s {
    int dev = -1;
    int N = 0, n = 0, K = 0, kinfo = 0, crc_len = 0, P = 0, systematic = 1;
    uint32_t crc_poly = 0;
    std::vector<uint8_t> frozen, punct;
    DevCode dc;
    void *d_blob = nullptr;
    std::mutex mu;
    std::map<std::vector<int>, Program> programs;
    // measured tuning per (list size, number format): warps per SM, fusion size
    std::map<int, Tuning> tune;
};

static uint32_t crc_poly32(int c, uint32_t poly)
{
    if (c == 0) return 0;
    uint32_t mask = c == 32 ? 0xFFFFFFFFu : ((1u << c) - 1u);
    return (poly & mask) << (32 - c);
}

extern "C" int pscl_create_code(int N, int K, const uint8_t *frozen, int crc_len, uint32_t crc_poly,
                                const uint8_t *puncture, int systematic, pscl_code *out)
{
    if (!out) return fail(PSCL_EINVAL, "out is NULL");
    *out = nullptr;
    if (N < 8 || N > (1 << kMaxLog2N) || (N & (N - 1)))
        return fail(PSCL_EINVAL, "N=%d: must be a power of two in [8, %d]", N, 1 << kMaxLog2N);
    if (!frozen) return fail(PSCL_EINVAL, "frozen is NULL");
    if (crc_len < 0 || crc_len > 32) return fail(PSCL_EINVAL, "crc_len=%d: must be 0..32", crc_len);
    if (crc_len > 0 && crc_len < 32 && (crc_poly >> crc_len) != 0)
        return fail(PSCL_EINVAL, "crc_poly 0x%x has bits above its %d-bit length", crc_poly, crc_len);
    int nf = 0;
    for (int i = 0; i < N; i++) nf += frozen[i] ? 1 : 0;
    if (N - nf != K || K < 1) return fail(PSCL_EINVAL, "K=%d but the frozen set leaves %d positions", K, N - nf);
    if (crc_len > K) return fail(PSCL_EINVAL, "crc_len=%d exceeds K=%d", crc_len, K);
    int P = 0;
    if (puncture)
        for (int i = 0; i < N; i++) P += puncture[i] ? 1 : 0;
    if (P >= N) return fail(PSCL_EINVAL, "every position is punctured");

    pscl_code_s *c = new pscl_code_s();
    c->N = N;
    c->n = 0;
    while ((1 << c->n) < N) c->n++;
    c->K = K;
    c->kinfo = K - crc_len;
    c->crc_len = crc_len;
    c->crc_poly = crc_poly;
    c->P = P;
    c->systematic = systematic ? 1 : 0;
    c->frozen.assign(frozen, frozen + N);
    for (auto &v : c->frozen) v = v ? 1 : 0;
    c->punct.assign(N, 0);
    if (puncture)
        for (int i = 0; i < N; i++) c->punct[i] = puncture[i] ? 1 : 0;

    // host images of the device arrays
    std::vector<int32_t> in_index(N);
    for (int i = 0, k = 0; i < N; i++) in_index[i] = c->punct[i] ? -1 : k++;
    std::vector<uint16_t> A;
    for (int i = 0; i < N; i++)
        if (!c->frozen[i]) A.push_back((uint16_t)i);
    const int NW = N >= 32 ? N / 32 : 1;
    std::vector<uint32_t> amask(NW, 0);
    for (int i = 0; i < N; i++)
        if (!c->frozen[i]) amask[i >> 5] |= 1u << (i & 31);
    std::vector<uint32_t> lut(256, 0);
    const uint32_t p32 = crc_poly32(crc_len, crc_poly);
    for (uint32_t b = 0; b < 256; b++) {
        uint32_t r = b << 24;
        for (int k = 0; k < 8; k++) r = (r & 0x80000000u) ? ((r << 1) ^ p32) : (r << 1);
        lut[b] = r;
    }
    // CRC check as a syndrome (Sec. IV-B): with the register starting at 0
    // the check "remainder of the first kinfo bits of u_A equals its last
    // crc_len bits" is linear over GF(2), so every position of A has a
    // crc_len-bit column and a path passes when the XOR of the columns of
    // its one-bits is 0.  Tabulated per codeword byte and byte value.
    const int NB = N >> 3;
    std::vector<uint32_t> syn((size_t)NB * 256, 0);
    if (crc_len > 0) {
        std::vector<uint32_t> poscol(N, 0);
        uint32_t r = p32;  // register after a lone one-bit at the last info index
        for (int k = c->kinfo - 1; k >= 0; --k) {
            poscol[A[k]] = r >> (32 - crc_len);
            r = (r & 0x80000000u) ? ((r << 1) ^ p32) : (r << 1);
        }
        for (int k = c->kinfo; k < K; ++k) poscol[A[k]] = 1u << (K - 1 - k);
        for (int q = 0; q < NB; ++q)
            for (int v = 0; v < 256; ++v) {
                uint32_t e = 0;
                for (int b = 0; b < 8; ++b)
                    if ((v >> b) & 1) e ^= poscol[8 * q + b];
                syn[(size_t)q * 256 + v] = e;
            }
    }
    // info-bit extraction per codeword byte: the byte's info positions (A
    // indices below K_info, increasing) are consecutive bits of the output
    std::vector<uint8_t> ext((size_t)NB * 256, 0);
    std::vector<uint16_t> ext_pos((size_t)NB + 1, 0);
    {
        std::vector<uint8_t> info_pos(N, 0);
        for (int k = 0; k < c->kinfo; ++k) info_pos[A[k]] = 1;
        int k = 0;
        for (int q = 0; q < NB; ++q) {
            ext_pos[q] = (uint16_t)k;
            for (int v = 0; v < 256; ++v) {
                uint32_t o = 0;
                int j = 0;
                for (int b = 0; b < 8; ++b)
                    if (info_pos[8 * q + b]) o |= (uint32_t)((v >> b) & 1) << j++;
                ext[(size_t)q * 256 + v] = (uint8_t)o;
            }
            for (int b = 0; b < 8; ++b) k += info_pos[8 * q + b];
        }
        ext_pos[NB] = (uint16_t)k;
    }
    size_t off_in = 0, off_A = off_in + 4 * (size_t)N, off_am = off_A + ((2 * (size_t)K + 15) & ~(size_t)15),
           off_lut = off_am + ((4 * (size_t)NW + 15) & ~(size_t)15), off_syn = off_lut + 1024,
           off_ext = off_syn + 4 * syn.size(), off_epos = off_ext + ext.size(),
           total = off_epos + ((2 * ext_pos.size() + 15) & ~(size_t)15);
    std::vector<uint8_t> blob(total, 0);
    memcpy(blob.data() + off_in, in_index.data(), 4 * (size_t)N);
    memcpy(blob.data() + off_A, A.data(), 2 * (size_t)K);
    memcpy(blob.data() + off_am, amask.data(), 4 * (size_t)NW);
    memcpy(blob.data() + off_lut, lut.data(), 1024);
    memcpy(blob.data() + off_syn, syn.data(), 4 * syn.size());
    memcpy(blob.data() + off_ext, ext.data(), ext.size());
    memcpy(blob.data() + off_epos, ext_pos.data(), 2 * ext_pos.size());
    cudaError_t e = cudaGetDevice(&c->dev);
    if (e == cudaSuccess) e = cudaMalloc(&c->d_blob, total);
    if (e == cudaSuccess) e = cudaMemcpy(c->d_blob, blob.data(), total, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        lib_free(c->d_blob);
        delete c;
        return fail(e == cudaErrorMemoryAllocation ? PSCL_ENOMEM : PSCL_ECUDA, "create_code: %s",
                    cudaGetErrorString(e));
    }
    char *base = (char *)c->d_blob;
    DevCode &dc = c->dc;
    dc.N = N;
    dc.n = c->n;
    dc.K = K;
    dc.kinfo = c->kinfo;
    dc.crc_len = crc_len;
    dc.systematic = c->systematic;
    dc.P = P;
    dc.poly32 = p32;
    dc.in_index = (const int32_t *)(base + off_in);
    dc.A = (const uint16_t *)(base + off_A);
    dc.amask = (const uint32_t *)(base + off_am);
    dc.crc_lut = (const uint32_t *)(base + off_lut);
    dc.syn = (const uint32_t *)(base + off_syn);
    dc.ext = (const uint8_t *)(base + off_ext);
    dc.ext_pos = (const uint16_t *)(base + off_epos);
    *out = c;
    return PSCL_OK;
}

extern "C" int pscl_destroy_code(pscl_code c)
{
    if (!c) return fail(PSCL_EINVAL, "code is NULL");
    for (auto &kv : c->programs) lib_free(kv.second.d_ops);
    lib_free(c->d_blob);
    delete c;
    return PSCL_OK;
}

extern "C" int pscl_code_info(pscl_code c, int *N, int *K, int *K_info, int *n_punctured)
{
    if (!c) return fail(PSCL_EINVAL, "code is NULL");
    if (N) *N = c->N;
    if (K) *K = c->K;
    if (K_info) *K_info = c->kinfo;
    if (n_punctured) *n_punctured = c->P;
    return PSCL_OK;
}

// ---------------------------------------------------------------------------
// node schedule (Sec. II-B tree pruning): pre-order traversal of Algorithm 1;
// a node whose leaves are all frozen (R0), all information (R1), all frozen
// but the last (REP) or only the first frozen (SPC) becomes one step when its
// type is enabled and within its size limits, the top-most such node winning;
// nodes below node_min leaves are decoded leaf by leaf.
static int classify(const pscl_code_s *c, const pscl_pruning *pr, int o, int S)
{
    int nf = 0;
    for (int i = o; i < o + S; i++) nf += c->frozen[i];
    if (S == 1) return nf ? NT_R0 : NT_R1;
    if (!pr || S < pr->node_min) return 0;
    if (nf == S && (pr->mask & PSCL_PRUNE_R0)) return NT_R0;
    if (nf == 0 && (pr->mask & PSCL_PRUNE_R1) && (pr->r1_max == 0 || S <= pr->r1_max)) return NT_R1;
    if (nf == S - 1 && !c->frozen[o + S - 1] && (pr->mask & PSCL_PRUNE_REP) && (pr->rep_max == 0 || S <= pr->rep_max))
        return NT_REP;
    if (nf == 1 && c->frozen[o] && S >= 4 && (pr->mask & PSCL_PRUNE_SPC) && (pr->spc_max == 0 || S <= pr->spc_max))
        return NT_SPC;
    return 0;
}

// defaults of the two tuning knobs: the largest subtree decoded in registers
// (2, 4 or 8 leaves; 1 = none; 0 = by format: 4 leaves in float, 2 in fixed
// point, the sizes the autotuner settles at for most codes) and the resident
// warps per SM the per-warp shared-memory slice is sized for; per code and
// (L, format) the autotuner's measurements override them (pscl_code_tune)
static int g_fuse_max = 0;
static int g_target_warps_per_sm = 32;  // with 28 resident: the rest of shared memory goes to L1

static int default_fuse(int quant)
{
    return g_fuse_max ? g_fuse_max : (quant == PSCL_F32 ? 4 : 2);
}

static int tune_key(int L, int quant, const pscl_pruning *pr)
{
    return L * 8 + quant + ((pr && pr->mask) ? 1024 : 0);
}

static const int kWarpsPerBlock = 4;  // default warps per block

static void tuning_for(pscl_code c, int L, int quant, const pscl_pruning *pr, int *wps, int *fuse, int *wpb = nullptr,
                       int *res = nullptr)
{
    *wps = g_target_warps_per_sm;
    *fuse = default_fuse(quant);
    if (wpb) *wpb = kWarpsPerBlock;
    if (res) *res = g_target_warps_per_sm;
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->tune.find(tune_key(L, quant, pr));
    if (it != c->tune.end()) {
        *wps = it->second.warps_per_sm;
        *fuse = it->second.fuse;
        if (wpb && it->second.warps_per_block > 0) *wpb = it->second.warps_per_block;
        if (res) *res = it->second.resident_warps > 0 ? it->second.resident_warps : it->second.warps_per_sm;
    }
}

// true when no node of the subtree of S leaves at o is a pruned node
static bool subtree_unpruned(const pscl_code_s *c, const pscl_pruning *pr, int o, int S)
{
    if (S == 1) return true;
    if (classify(c, pr, o, S)) return false;
    return subtree_unpruned(c, pr, o, S / 2) && subtree_unpruned(c, pr, o + S / 2, S / 2);
}

static int gen_program(const pscl_code_s *c, const pscl_pruning *pr, int fuse, bool quad, int d, int o, int S,
                       int side, std::vector<uint32_t> &ops, int &max_depth)
{
    int type = classify(c, pr, o, S);
    if (type) {
        int t = 0;
        if (type == NT_R1) {
            int r1t = pr ? pr->r1_t : 1;
            t = S == 1 ? 1 : (r1t < S ? r1t : S);
            if (t < 1 || t > 3) return fail(PSCL_EUNSUPPORTED, "R1 flip depth %d (node size %d) outside 1..3", t, S);
        } else if (type == NT_SPC) {
            t = pr->spc_t < S ? pr->spc_t : S;
            if (t < 1 || t > 4) return fail(PSCL_EUNSUPPORTED, "SPC flip depth %d (node size %d) outside 1..4", t, S);
        }
        ops.push_back(op_make(OP_NODE, (uint32_t)d, (uint32_t)type, (uint32_t)side, (uint32_t)t));
        if (d > max_depth) max_depth = d;
        return PSCL_OK;
    }
    if (d >= 1 && S <= fuse && subtree_unpruned(c, pr, o, S)) {
        // the whole subtree is decoded in registers by one step
        uint32_t fz = 0;
        for (int i = 0; i < S; i++) fz |= (uint32_t)c->frozen[o + i] << i;
        ops.push_back(op_make(OP_RSUB, (uint32_t)d, 0, (uint32_t)side, 0) | (fz << 16));
        if (d > max_depth) max_depth = d;
        return PSCL_OK;
    }
    if (quad && d >= 1 && fuse == 4 && S == 16 && subtree_unpruned(c, pr, o, S)) {
        // two levels of register-subtree pairs in one step (measured faster
        // than separate steps for 4-leaf subtrees only)
        uint32_t fz = 0;
        for (int i = 0; i < S; i++) fz |= (uint32_t)c->frozen[o + i] << i;
        ops.push_back(op_make(OP_RSUB4, (uint32_t)d, 0, (uint32_t)side, 0) | (fz << 16));
        if (d > max_depth) max_depth = d;
        return PSCL_OK;
    }
    if (d >= 1 && fuse >= 2 && S == 2 * fuse && subtree_unpruned(c, pr, o, S)) {
        // f, both register subtrees, g and h in one step
        uint32_t fz = 0;
        for (int i = 0; i < S; i++) fz |= (uint32_t)c->frozen[o + i] << i;
        ops.push_back(op_make(OP_RSUB2, (uint32_t)d, 0, (uint32_t)side, 0) | (fz << 16));
        if (d > max_depth) max_depth = d;
        return PSCL_OK;
    }
    ops.push_back(op_make(OP_F, (uint32_t)d, 0, 0, 0));
    int rc = gen_program(c, pr, fuse, quad, d + 1, o, S / 2, 0, ops, max_depth);
    if (rc) return rc;
    ops.push_back(op_make(OP_G, (uint32_t)d, 0, 0, 0));
    rc = gen_program(c, pr, fuse, quad, d + 1, o + S / 2, S / 2, 1, ops, max_depth);
    if (rc) return rc;
    if (d > 0) ops.push_back(op_make(OP_COMB, (uint32_t)(d + 1), 0, (uint32_t)side, 0));
    return PSCL_OK;
}

// The schedule of the one-path (SC) kernel: the same pruned tree without
// register subtrees; every step carries its node's leaf offset in bits
// 16..31 (an h step the offset of the node it completes).
// Subtrees of up to kScFuse leaves are one step (OP_RSUB, decoded in
// registers; the kernel reads their frozen leaves from the code's mask and,
// when the step's t field is 1, the pruned nodes inside them from the
// node-type words stored after the schedule, see sc_node_types).
constexpr int kScFuse = 16;

static void gen_sc_program(const pscl_code_s *c, const pscl_pruning *pr, int d, int o, int S, int side,
                           std::vector<uint32_t> &ops, int &max_depth)
{
    const uint32_t off = (uint32_t)o << 16;
    int type = classify(c, pr, o, S);
    if (type) {
        ops.push_back(op_make(OP_NODE, (uint32_t)d, (uint32_t)type, (uint32_t)side, 0) | off);
        if (d > max_depth) max_depth = d;
        return;
    }
    if (d >= 1 && S <= kScFuse) {
        const uint32_t t = subtree_unpruned(c, pr, o, S) ? 0u : 1u;  // 1: pruned nodes inside
        ops.push_back(op_make(OP_RSUB, (uint32_t)d, 0, (uint32_t)side, t) | off);
        if (d > max_depth) max_depth = d;
        return;
    }
    if (d >= 1 && S == 2 * kScFuse) {
        // f, both register subtrees, g and h as one step; t bits: pruned
        // nodes inside the left / right half
        const uint32_t t = (subtree_unpruned(c, pr, o, S / 2) ? 0u : 1u) |
                           (subtree_unpruned(c, pr, o + S / 2, S / 2) ? 0u : 2u);
        ops.push_back(op_make(OP_RSUB2, (uint32_t)d, 0, (uint32_t)side, t) | off);
        if (d > max_depth) max_depth = d;
        return;
    }
    ops.push_back(op_make(OP_F, (uint32_t)d, 0, 0, 0) | off);
    gen_sc_program(c, pr, d + 1, o, S / 2, 0, ops, max_depth);
    ops.push_back(op_make(OP_G, (uint32_t)d, 0, 0, 0) | off);
    gen_sc_program(c, pr, d + 1, o + S / 2, S / 2, 1, ops, max_depth);
    if (d > 0) ops.push_back(op_make(OP_COMB, (uint32_t)(d + 1), 0, (uint32_t)side, 0) | off);
}

// Node types inside the SC kernel's register subtrees: for each group of 16
// leaves (g = 0 .. ceil(N/16) - 1) one 64-bit word holding, for the group's
// nodes of 2..16 leaves in heap order (node h = 1 .. 15: size 16 >> floor(log2
// h), offset g*16 + (h - 2^floor(log2 h)) * size), the pruned-node type at
// bits 3(h-1) (0: not a pruned node); appended to the schedule as pairs of
// 32-bit words from an even index.
static void sc_node_types(const pscl_code_s *c, const pscl_pruning *pr, std::vector<uint32_t> &ops)
{
    if (ops.size() & 1) ops.push_back(0u);
    const int groups = (c->N + 15) / 16;
    for (int g = 0; g < groups; g++) {
        uint64_t w = 0;
        for (int h = 1; h < 16; h++) {
            int l = 0;
            while ((2 << l) <= h) l++;
            const int S = 16 >> l, o = g * 16 + (h - (1 << l)) * S;
            if (o + S > c->N) continue;
            w |= (uint64_t)classify(c, pr, o, S) << (3 * (h - 1));
        }
        ops.push_back((uint32_t)w);
        ops.push_back((uint32_t)(w >> 32));
    }
}

// Peephole fusion of the schedule: a right register-subtree pair (or quad)
// directly followed by its parent's h step takes that step over.
static void fuse_ops(std::vector<uint32_t> &ops)
{
    std::vector<uint32_t> out;
    out.reserve(ops.size());
    for (size_t i = 0; i < ops.size(); i++) {
        const uint32_t a = ops[i];
        if (i + 1 < ops.size()) {
            const uint32_t b = ops[i + 1];
            if ((op_code(a) == OP_RSUB2 || op_code(a) == OP_RSUB4) && op_side(a) == 1 && op_code(b) == OP_COMB &&
                op_depth(b) == op_depth(a)) {
                out.push_back(a | ((1u | ((uint32_t)op_side(b) << 1)) << 12));
                i++;
                continue;
            }
        }
        out.push_back(a);
    }
    ops.swap(out);
}

// Schedules depend on the pruning, the fusion size and whether the number
// format is float (the 16-leaf quad step is used for float only: the
// fixed-point kernels measured slower with it)
static std::vector<int> prune_key(const pscl_pruning *pr, int fuse, bool fixed)
{
    if (!pr || pr->mask == 0) return {fuse, fixed ? 1 : 0, 0};
    return {fuse, fixed ? 1 : 0, (int)pr->mask, pr->rep_max, pr->spc_max, pr->r1_t, pr->spc_t, pr->r1_max,
            pr->node_min};
}

static int check_pruning(const pscl_pruning *pr)
{
    if (!pr || pr->mask == 0) return PSCL_OK;
    if (pr->mask & ~15u) return fail(PSCL_EINVAL, "pruning mask 0x%x has unknown bits", pr->mask);
    if (pr->rep_max < 0 || pr->spc_max < 0 || pr->r1_max < 0 || pr->node_min < 0)
        return fail(PSCL_EINVAL, "negative pruning size limit");
    if ((pr->mask & PSCL_PRUNE_R1) && (pr->r1_t < 1 || pr->r1_t > 3))
        return fail(PSCL_EUNSUPPORTED, "r1_t=%d: the kernels support 1..3", pr->r1_t);
    if ((pr->mask & PSCL_PRUNE_SPC) && (pr->spc_t < 1 || pr->spc_t > 4))
        return fail(PSCL_EUNSUPPORTED, "spc_t=%d: the kernels support 1..4", pr->spc_t);
    return PSCL_OK;
}

static int get_program(pscl_code c, const pscl_pruning *pr, int fuse, bool fixed, Program *out)
{
    int rc = check_pruning(pr);
    if (rc) return rc;
    const pscl_pruning *eff = (pr && pr->mask) ? pr : nullptr;
    std::vector<int> key = prune_key(pr, fuse, fixed);
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->programs.find(key);
    if (it != c->programs.end()) {
        *out = it->second;
        return PSCL_OK;
    }
    std::vector<uint32_t> ops;
    int max_depth = 0;
    if (fuse == 0) {
        gen_sc_program(c, eff, 0, 0, c->N, 1, ops, max_depth);  // the one-path kernel's schedule
    } else {
        rc = gen_program(c, eff, fuse, !fixed, 0, 0, c->N, 1, ops, max_depth);
        if (rc) return rc;
    }
    if (fuse != 0 && max_depth > kTabLayers)
        return fail(PSCL_EUNSUPPORTED,
                    "N=%d with register subtrees of %d leaf(s): the schedule reaches depth %d, the kernels' slot "
                    "tables hold %d layers (use subtrees of 2 or more leaves)",
                    c->N, fuse, max_depth, kTabLayers);
    if (fuse != 0) fuse_ops(ops);
    Program p;
    p.n_ops = (int)ops.size();
    p.max_depth = max_depth;
    p.root_special = (op_code(ops[0]) == OP_NODE) ? 1 : 0;
    for (uint32_t w : ops)
        if (op_code(w) == OP_NODE) p.has_nodes = 1;
    if (fuse == 0) sc_node_types(c, eff, ops);  // after the n_ops schedule steps
    CU(cudaMalloc(&p.d_ops, ops.size() * sizeof(uint32_t)));
    cudaError_t e = cudaMemcpy(p.d_ops, ops.data(), ops.size() * sizeof(uint32_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        lib_free(p.d_ops);
        return fail(PSCL_ECUDA, "program upload: %s", cudaGetErrorString(e));
    }
    c->programs[key] = p;
    *out = p;
    return PSCL_OK;
}

// lookup of an already prepared schedule; never builds or allocates
static int find_program(pscl_code c, const pscl_pruning *pr, int fuse, bool fixed, Program *out)
{
    int rc = check_pruning(pr);
    if (rc) return rc;
    std::vector<int> key = prune_key(pr, fuse, fixed);
    std::lock_guard<std::mutex> lk(c->mu);
    auto it = c->programs.find(key);
    if (it == c->programs.end())
        return fail(PSCL_EINVAL, "no node schedule for this pruning setting: call pscl_prepare first");
    *out = it->second;
    return PSCL_OK;
}

extern "C" int pscl_prepare(pscl_code c, const pscl_pruning *pr)
{
    if (!c) return fail(PSCL_EINVAL, "code is NULL");
    // the default schedule and every fusion size the code's tuning uses
    // 0: the one-path (SC) kernel's schedule
    std::vector<int> fuses = {default_fuse(PSCL_F32), default_fuse(PSCL_I16), 0};
    {
        std::lock_guard<std::mutex> lk(c->mu);
        for (auto &kv : c->tune) fuses.push_back(kv.second.fuse);
    }
    for (int f : fuses)
        for (int fixed = 0; fixed < 2; ++fixed) {
            Program p;
            int rc = get_program(c, pr, f, fixed != 0, &p);
            if (rc) return rc;
        }
    return PSCL_OK;
}

extern "C" int pscl_code_tune(pscl_code c, int L, pscl_quant quant, const pscl_pruning *pruning, int warps_per_sm,
                              int fuse_leaves, int warps_per_block, int resident_warps)
{
    if (!c) return fail(PSCL_EINVAL, "code is NULL");
    if (L != 1 && L != 2 && L != 4 && L != 8 && L != 16 && L != 32) return fail(PSCL_EINVAL, "L=%d", L);
    if (quant < PSCL_F32 || quant > PSCL_I8) return fail(PSCL_EINVAL, "unknown quantisation %d", (int)quant);
    std::lock_guard<std::mutex> lk(c->mu);
    if (warps_per_sm == 0 && fuse_leaves == 0) {
        c->tune.erase(tune_key(L, (int)quant, pruning));
        return PSCL_OK;
    }
    if (warps_per_sm < 1 || warps_per_sm > 64) return fail(PSCL_EINVAL, "warps per SM %d out of 1..64", warps_per_sm);
    if (resident_warps < 0 || resident_warps > 64)
        return fail(PSCL_EINVAL, "resident warps %d out of 0..64", resident_warps);
    if (fuse_leaves != 1 && fuse_leaves != 2 && fuse_leaves != 4 && fuse_leaves != 8)
        return fail(PSCL_EINVAL, "fusion size %d: must be 1, 2, 4 or 8", fuse_leaves);
    if (warps_per_block != 0 && warps_per_block != 1 && warps_per_block != 2 && warps_per_block != 4 &&
        warps_per_block != 8)
        return fail(PSCL_EINVAL, "warps per block %d: must be 1, 2, 4 or 8 (0 = default)", warps_per_block);
    Tuning t;
    t.warps_per_sm = warps_per_sm;
    t.fuse = fuse_leaves;
    t.warps_per_block = warps_per_block;
    t.resident_warps = resident_warps;
    c->tune[tune_key(L, (int)quant, pruning)] = t;
    return PSCL_OK;
}

// ---------------------------------------------------------------------------
// per-warp memory layout: every buffer goes to shared memory while the budget
// lasts, deepest (smallest, most often touched) layers first; the rest lives
// in the warp's global scratch slice.
static void make_layout(const pscl_code_s *c, const Program &pg, int L, int quant, size_t smem_budget, Layout *lay)
{
    memset(lay, 0, sizeof(*lay));
    const int EPW = quant == PSCL_F32 ? 1 : (quant == PSCL_I16 ? 2 : 4);
    const int fpw = 32 / L;
    uint32_t so = 0, go = 0;
    auto align16 = [](uint32_t v) { return (v + 15u) & ~15u; };
    // the warp's copy of its Item, then the selection scatter (64 words) and
    // frame ids (32 words)
    lay->src_off = kItemBytes + kPtabBytes;
    lay->info_words = (uint32_t)std::max(64, (c->kinfo + 31) / 32);
    so = align16(lay->src_off + (lay->info_words + 32) * 4);
    const int maxd = pg.max_depth;
    for (int d = maxd; d >= 0; d--) {
        const int S = c->N >> d;
        const uint32_t rows = (uint32_t)((S + EPW - 1) / EPW);
        // words of a path are stored in groups of four (16-byte accesses)
        const uint32_t words = ((rows + 3u) / 4u) * 4u * (uint32_t)(d == 0 ? fpw : 32);
        const uint32_t bwords = (uint32_t)(S >= 32 ? S / 32 : 1) * 32u;
        // LLR layer d
        lay->llr_words[d] = words;
        if (so + words * 4 <= smem_budget) {
            lay->llr_off[d] = so;
            lay->llr_smem |= 1u << d;
            so = align16(so + words * 4);
        } else {
            lay->llr_off[d] = go;
            go = align16(go + words * 4);
        }
        // partial-sum buffers: BL_d, BR_d for d >= 1; BR_0 when the root is a node
        lay->b_words[d] = bwords;
        const bool need_bl = d >= 1, need_br = d >= 1 || pg.root_special;
        if (need_bl) {
            if (so + bwords * 4 <= smem_budget) {
                lay->bl_off[d] = so;
                lay->bl_smem |= 1u << d;
                so = align16(so + bwords * 4);
            } else {
                lay->bl_off[d] = go;
                go = align16(go + bwords * 4);
            }
        }
        if (need_br) {
            if (so + bwords * 4 <= smem_budget) {
                lay->br_off[d] = so;
                lay->br_smem |= 1u << d;
                so = align16(so + bwords * 4);
            } else {
                lay->br_off[d] = go;
                go = align16(go + bwords * 4);
            }
        }
    }
    if (!c->systematic) {
        lay->ns_words = (uint32_t)(c->N >= 32 ? c->N / 32 : 1) * 32u;
        lay->ns_off = go;
        go = align16(go + lay->ns_words * 4);
    }
    lay->smem_per_warp = so;
    lay->gmem_per_warp = (go + 255u) & ~255u;
}

// Shared-memory slice of the one-path (SC) kernel's warp: the partial-sum
// bits (N bits), LLR layers 1..max_depth (layer d: N/2^d values), and the
// info-bit buffer.  Nothing lives in global scratch.
static void make_sc_layout(const pscl_code_s *c, const Program &pg, int quant, Layout *lay)
{
    memset(lay, 0, sizeof(*lay));
    const int EPW = quant == PSCL_F32 ? 1 : (quant == PSCL_I16 ? 2 : 4);
    auto align16 = [](uint32_t v) { return (v + 15u) & ~15u; };
    uint32_t so = 0;
    lay->bl_off[0] = so;
    lay->b_words[0] = (uint32_t)(c->N >= 32 ? c->N / 32 : 1);
    so = align16(so + lay->b_words[0] * 4);
    for (int d = 1; d <= pg.max_depth; d++) {
        const int S = c->N >> d;
        const uint32_t words = (uint32_t)(((S + EPW - 1) / EPW + 3) / 4 * 4);
        lay->llr_off[d] = so;
        lay->llr_words[d] = words;
        lay->llr_smem |= 1u << d;
        so = align16(so + words * 4);
    }
    lay->info_words = (uint32_t)std::max(1, (c->kinfo + 31) / 32);
    lay->src_off = so;
    so = align16(so + lay->info_words * 4);
    lay->smem_per_warp = so;
    lay->gmem_per_warp = 0;
}

// one-path stages (SC, the first stage of FA and PA) of batches of up to
// kScQuarterWaves[float, fixed] / 4 waves of resident warps use the SC
// kernel (measured crossovers with the list kernel on (2048,1723) at 4.5 dB:
// about 6 waves in float, between 2 and 3 in fixed point)
static bool g_sc_kernel = true;
constexpr long long kScQuarterWaves[2] = {24, 10};

// ---------------------------------------------------------------------------
// launch plan for one decode call
struct Plan {
    Program pg;
    Layout lay;
    int warps_per_block = 4;
    int grid = 0;
    int total_warps = 0;
    size_t smem_block = 0;
    size_t gmem_scratch = 0;   // per-warp slices
    uint32_t gmem_per_warp = 0;
    size_t list_bytes = 0;     // adaptive frame lists + counters
    size_t total_ws = 0;
    int n_stages = 0;
    int stages[8];
    size_t budget = 0;         // shared-memory bytes per warp
    int kv = KV_PLAIN;         // decoder kernel variant
    // one-path stage on the SC kernel (warp per frame, all state on chip)
    bool sc = false;
    Program sc_pg;
    Layout sc_lay;
    int sc_grid = 0, sc_total_warps = 0;
};

// shared-memory bytes per warp when wps warps (in blocks of wpb) share an
// SM: each block gets an equal share of the SM's shared memory, less the
// runtime's per-block reservation, rounded down to the 128-byte allocation
// unit, split over its warps
static size_t slice_budget(const DevProps &dp, int wps, int wpb = kWarpsPerBlock)
{
    const int blocks = (wps + wpb - 1) / wpb;
    const long long per_block = (long long)dp.smem_per_sm / blocks - dp.smem_reserved;
    size_t budget = per_block > 0 ? ((size_t)per_block & ~(size_t)127) / wpb : 0;
    if (budget > (size_t)dp.smem_optin / wpb) budget = (size_t)dp.smem_optin / wpb;
    return budget & ~(size_t)15;
}

static int make_plan(pscl_code c, int n_frames, int L, pscl_algo algo, const pscl_pruning *pr, pscl_quant quant,
                     Plan *pl, bool build_program = true)
{
    if (!c) return fail(PSCL_EINVAL, "code is NULL");
    if (n_frames < 0) return fail(PSCL_EINVAL, "n_frames=%d", n_frames);
    if (L != 1 && L != 2 && L != 4 && L != 8 && L != 16 && L != 32)
        return fail(PSCL_EINVAL, "L=%d: must be 1, 2, 4, 8, 16 or 32", L);
    if (algo < PSCL_SC || algo > PSCL_FASCL) return fail(PSCL_EINVAL, "unknown algorithm %d", (int)algo);
    if (quant < PSCL_F32 || quant > PSCL_I8) return fail(PSCL_EINVAL, "unknown quantisation %d", (int)quant);
    int dev;
    CU(cudaGetDevice(&dev));
    if (dev != c->dev) return fail(PSCL_EINVAL, "code was created on device %d, current device is %d", c->dev, dev);
    int wps, fuse, wpb, res;
    tuning_for(c, L, (int)quant, pr, &wps, &fuse, &wpb, &res);
    pl->warps_per_block = wpb;
    const bool fixed = quant != PSCL_F32;
    int rc = build_program ? get_program(c, pr, fuse, fixed, &pl->pg) : find_program(c, pr, fuse, fixed, &pl->pg);
    if (rc) return rc;
    DevProps dp;
    rc = get_props(&dp);
    if (rc) return rc;
    // stages of the algorithm
    pl->n_stages = 0;
    if (algo == PSCL_SC) pl->stages[pl->n_stages++] = 1;
    else if (algo == PSCL_CASCL) pl->stages[pl->n_stages++] = L;
    else if (algo == PSCL_FASCL) {
        for (int l = 1; l < L; l *= 2) pl->stages[pl->n_stages++] = l;
        pl->stages[pl->n_stages++] = L;
    } else {
        pl->stages[pl->n_stages++] = 1;
        if (L > 1) pl->stages[pl->n_stages++] = L;
    }
    // layout: the largest stage list size determines frames per warp, but
    // every stage uses the same per-warp slices (the layout of the smallest
    // list size needs the most layer-0 room, the largest the most paths:
    // both only depend on N, EPW and 32/L for layer 0)
    const size_t budget = slice_budget(dp, wps, wpb);
    pl->budget = budget;
    // each stage recomputes its own layout at launch; the plan keeps maxima
    uint32_t max_smem = 0, max_gmem = 0;
    for (int s = 0; s < pl->n_stages; s++) {
        Layout l;
        make_layout(c, pl->pg, pl->stages[s], (int)quant, budget, &l);
        if (l.smem_per_warp > max_smem) max_smem = l.smem_per_warp;
        if (l.gmem_per_warp > max_gmem) max_gmem = l.gmem_per_warp;
    }
    pl->smem_block = (size_t)max_smem * wpb;
    int bps = 0;
    pl->kv = kernel_variant(pl->pg.has_nodes != 0, res);
    cudaError_t e = scl_func_attrs((int)quant, pl->kv, pl->smem_block, 32 * wpb, &bps);
    if (e != cudaSuccess) return fail(PSCL_ECUDA, "kernel attributes: %s", cudaGetErrorString(e));
    if (bps < 1) return fail(PSCL_EUNSUPPORTED, "no block fits (shared memory %zu bytes)", pl->smem_block);
    const int max_warps = dp.sms * bps * wpb;
    const int fpw_min = 32 / pl->stages[pl->n_stages - 1];
    long long tasks = ((long long)n_frames + fpw_min - 1) / fpw_min;
    long long want = tasks < 1 ? 1 : tasks;
    // the first stage may have more frames per warp; size the grid for the
    // stage with the most tasks
    long long tasks0 = ((long long)n_frames + (32 / pl->stages[0]) - 1) / (32 / pl->stages[0]);
    if (tasks0 > want) want = tasks0;
    int tw = (int)(want < max_warps ? want : max_warps);
    pl->grid = (tw + wpb - 1) / wpb;
    pl->total_warps = pl->grid * wpb;
    pl->gmem_per_warp = max_gmem;
    pl->gmem_scratch = (size_t)max_gmem * (size_t)pl->total_warps;
    pl->list_bytes = pl->n_stages > 1 ? (2 * (size_t)n_frames * 4 + 256 + 255) & ~(size_t)255 : 0;
    pl->total_ws = 256 /* error word + counters */ + pl->list_bytes + pl->gmem_scratch;
    // a first stage with one path runs on the SC kernel
    pl->sc = false;
    if (g_sc_kernel && pl->stages[0] == 1) {
        rc = build_program ? get_program(c, pr, 0, fixed, &pl->sc_pg) : find_program(c, pr, 0, fixed, &pl->sc_pg);
        if (rc) return rc;
        make_sc_layout(c, pl->sc_pg, (int)quant, &pl->sc_lay);
        int sbps = 0;
        const size_t sblock = (size_t)pl->sc_lay.smem_per_warp * kWarpsPerBlock;
        e = sc_attrs((int)quant, sblock, 32 * kWarpsPerBlock, &sbps);
        if (e != cudaSuccess) return fail(PSCL_ECUDA, "SC kernel attributes: %s", cudaGetErrorString(e));
        // A warp spends far more instructions per frame than a lane of the
        // list kernel, which decodes 32 one-path frames per warp side by side,
        // but it finishes its frame about five times sooner: the SC kernel
        // takes batches of up to a few waves of resident warps, where it
        // finishes first; larger batches go to the list kernel.
        const long long smax = (long long)dp.sms * sbps * kWarpsPerBlock;
        if (sbps >= 1 && 4 * (long long)n_frames <= kScQuarterWaves[fixed ? 1 : 0] * smax) {
            const long long sw = n_frames < 1 ? 1 : (n_frames < smax ? n_frames : smax);
            pl->sc_grid = (int)((sw + kWarpsPerBlock - 1) / kWarpsPerBlock);
            pl->sc_total_warps = pl->sc_grid * kWarpsPerBlock;
            pl->sc = true;
        }
    }
    return PSCL_OK;
}

extern "C" int pscl_workspace_size(pscl_code c, int n_frames, int L, pscl_algo algo, const pscl_pruning *pr,
                                   pscl_quant quant, size_t *bytes)
{
    if (!bytes) return fail(PSCL_EINVAL, "bytes is NULL");
    Plan pl;
    int rc = make_plan(c, n_frames, L, algo, pr, quant, &pl);
    if (rc) return rc;
    *bytes = pl.total_ws;
    return PSCL_OK;
}

#ifdef PSCL_OPPROF
// step-profiling build: one counter block per device, zeroed at allocation
static std::mutex g_prof_mu;
static std::map<int, unsigned long long *> g_prof;
static unsigned long long *prof_buffer()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    auto it = g_prof.find(dev);
    if (it != g_prof.end()) return it->second;
    unsigned long long *p = nullptr;
    if (cudaMalloc(&p, 32 * sizeof(unsigned long long)) != cudaSuccess) return nullptr;
    cudaMemset(p, 0, 32 * sizeof(unsigned long long));
    g_prof[dev] = p;
    return p;
}
#endif

static cudaError_t launch_stage(int quant, int kv, const KParams &kp, int grid, size_t smem, cudaStream_t s,
                                int wpb = kWarpsPerBlock)
{
#ifdef PSCL_OPPROF
    KParams kq = kp;
    kq.op_cycles = prof_buffer();
    return launch_scl(quant, kv, kq, grid, 32 * wpb, smem, s);
#else
    return launch_scl(quant, kv, kp, grid, 32 * wpb, smem, s);
#endif
}

static int g_last_launches = 0;

static int run_decode(pscl_code c, const float *llr, int n_frames, int L, pscl_algo algo, const pscl_pruning *pr,
                      pscl_quant quant, uint8_t *info_out, int32_t *status_out, float *pm_out, void *ws,
                      size_t ws_bytes, cudaStream_t stream, const Plan &pl)
{
    if (n_frames == 0) return PSCL_OK;
    if (!llr || !info_out || !status_out) return fail(PSCL_EINVAL, "llr, info_out and status_out are required");
    if (ws_bytes < pl.total_ws || !ws) return fail(PSCL_EINVAL, "workspace too small: %zu < %zu", ws_bytes, pl.total_ws);
    if (((uintptr_t)ws) & 255u) return fail(PSCL_EINVAL, "workspace must be 256-byte aligned");
    char *w = (char *)ws;
    uint32_t *err = (uint32_t *)w;
    int32_t *counts = (int32_t *)(w + 64);  // two list counters
    int32_t *lists = (int32_t *)(w + 256);
    char *gmem = w + 256 + pl.list_bytes;
    const size_t budget = pl.budget;
    int launches = 0;
    for (int s = 0; s < pl.n_stages; s++) {
        const int Ls = pl.stages[s];
        KParams kp;
        memset(&kp, 0, sizeof(kp));
        Item &it = kp.single;
        it.code = c->dc;
        it.ops = pl.pg.d_ops;
        it.n_ops = pl.pg.n_ops;
        it.root_special = pl.pg.root_special;
        make_layout(c, pl.pg, Ls, (int)quant, budget, &it.lay);
        it.llr = llr;
        it.n_frames = n_frames;
        it.L = Ls;
        it.L_out = L;
        it.stage_L = Ls;
        it.info_out = info_out;
        it.status_out = status_out;
        it.pm_out = pm_out;
        it.err = err;
        kp.gmem = gmem;
        kp.gmem_per_warp = pl.gmem_per_warp;
        kp.smem_per_warp = it.lay.smem_per_warp;
        kp.total_warps = pl.total_warps;
        const bool last = s == pl.n_stages - 1;
        if (s > 0) {
            it.frame_list = lists + (size_t)((s - 1) & 1) * (size_t)n_frames;
            it.list_count = counts + ((s - 1) & 1);
        }
        if (!last) {
            it.next_list = lists + (size_t)(s & 1) * (size_t)n_frames;
            it.next_count = counts + (s & 1);
            CU(cudaMemsetAsync(it.next_count, 0, sizeof(int32_t), stream));
        }
        cudaError_t e;
        if (s == 0 && pl.sc) {
            // one path: warp per frame, layers and partial sums on chip
            it.ops = pl.sc_pg.d_ops;
            it.n_ops = pl.sc_pg.n_ops;
            it.root_special = pl.sc_pg.root_special;
            it.lay = pl.sc_lay;
            kp.smem_per_warp = pl.sc_lay.smem_per_warp;
            kp.total_warps = pl.sc_total_warps;
            kp.gmem = nullptr;
            kp.gmem_per_warp = 0;
            e = launch_sc((int)quant, kp, pl.sc_grid, 32 * kWarpsPerBlock,
                          (size_t)pl.sc_lay.smem_per_warp * kWarpsPerBlock, stream);
        } else {
            const size_t smem = (size_t)it.lay.smem_per_warp * pl.warps_per_block;
            e = launch_stage((int)quant, pl.kv, kp, pl.grid, smem, stream, pl.warps_per_block);
        }
        if (e != cudaSuccess) return fail(PSCL_ECUDA, "decode launch: %s", cudaGetErrorString(e));
        launches++;
    }
    g_last_launches = launches;
    return PSCL_OK;
}

// library-owned workspaces, one per (device, stream), grown on demand: calls
// on one stream run in stream order and may share theirs, calls on different
// streams never share one
static std::map<std::pair<int, void *>, std::pair<void *, size_t>> g_ws;

// the library's workspace of (device, stream), grown to at least `bytes`
static int stream_workspace(int dev, void *stream, size_t bytes, void **ws, size_t *wsb)
{
    std::lock_guard<std::mutex> lk(g_mu);
    auto &slot = g_ws[std::make_pair(dev, stream)];
    if (slot.second < bytes) {
        if (slot.first) {
            // only this stream's queued work can still use the old one
            CU(cudaStreamSynchronize((cudaStream_t)stream));
            lib_free(slot.first);
            slot.first = nullptr;
            slot.second = 0;
        }
        size_t want = bytes + bytes / 4;
        CU(cudaMalloc(&slot.first, want));
        CU(cudaMemset(slot.first, 0, 256));
        slot.second = want;
    }
    *ws = slot.first;
    *wsb = slot.second;
    return PSCL_OK;
}

extern "C" int pscl_decode(pscl_code c, const float *llr, int n_frames, int L, pscl_algo algo,
                           const pscl_pruning *pr, pscl_quant quant, uint8_t *info_out, int32_t *status_out,
                           float *pm_out, void *stream)
{
    Plan pl;
    int rc = make_plan(c, n_frames, L, algo, pr, quant, &pl);
    if (rc) return rc;
    int dev;
    CU(cudaGetDevice(&dev));
    void *ws;
    size_t wsb;
    rc = stream_workspace(dev, stream, pl.total_ws, &ws, &wsb);
    if (rc) return rc;
    return run_decode(c, llr, n_frames, L, algo, pr, quant, info_out, status_out, pm_out, ws, wsb,
                      (cudaStream_t)stream, pl);
}

// ---------------------------------------------------------------------------
// Decode from host buffers (pscl_decode_host): the batch is cut into up to
// kHostChunks chunks; one internal stream copies the chunks' LLRs in, two
// decode them alternately (each with its own workspace) and copy their
// outputs back, so copies and decodes of different chunks overlap, and a
// chunk's decode may start while the previous one drains.  Per (device,
// caller stream): the streams, events and a device staging buffer.
constexpr int kHostChunks = 4;
constexpr int kHostMinChunk = 4096;  // frames: smaller batches are not cut
struct HostCtx {
    cudaStream_t copy = nullptr;
    cudaStream_t comp[2] = {nullptr, nullptr};
    cudaEvent_t ev_start = nullptr, ev_done[2] = {nullptr, nullptr}, ev_in[kHostChunks] = {};
    void *dbuf = nullptr;
    size_t dbytes = 0;
};
static std::map<std::pair<int, void *>, HostCtx> g_host;

static int host_ctx(int dev, void *stream, size_t bytes, HostCtx **out)
{
    std::lock_guard<std::mutex> lk(g_mu);
    HostCtx &h = g_host[std::make_pair(dev, stream)];
    if (!h.copy) {
        CU(cudaStreamCreateWithFlags(&h.copy, cudaStreamNonBlocking));
        CU(cudaStreamCreateWithFlags(&h.comp[0], cudaStreamNonBlocking));
        CU(cudaStreamCreateWithFlags(&h.comp[1], cudaStreamNonBlocking));
        CU(cudaEventCreateWithFlags(&h.ev_start, cudaEventDisableTiming));
        for (auto &e : h.ev_done) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        for (auto &e : h.ev_in) CU(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    if (h.dbytes < bytes) {
        if (h.dbuf) {
            // earlier calls' copies and decodes may still use it
            CU(cudaStreamSynchronize(h.copy));
            CU(cudaStreamSynchronize(h.comp[0]));
            CU(cudaStreamSynchronize(h.comp[1]));
            lib_free(h.dbuf);
            h.dbuf = nullptr;
            h.dbytes = 0;
        }
        const size_t want = bytes + bytes / 4;
        CU(cudaMalloc(&h.dbuf, want));
        h.dbytes = want;
    }
    *out = &h;
    return PSCL_OK;
}

extern "C" int pscl_decode_host(pscl_code c, const float *llr_host, int n_frames, int L, pscl_algo algo,
                                const pscl_pruning *pr, pscl_quant quant, uint8_t *info_host,
                                int32_t *status_host, void *stream)
{
    // every argument error is reported before anything is enqueued
    Plan pl;
    int rc = make_plan(c, n_frames, L, algo, pr, quant, &pl);
    if (rc) return rc;
    if (n_frames == 0) return PSCL_OK;
    if (!llr_host || !info_host || !status_host)
        return fail(PSCL_EINVAL, "llr_host, info_host and status_host are required");
    int dev;
    CU(cudaGetDevice(&dev));
    const size_t row = (size_t)(c->N - c->P), nb = (size_t)((c->kinfo + 7) / 8);
    auto up = [](size_t v) { return (v + 255) & ~(size_t)255; };
    const size_t off_info = up((size_t)n_frames * row * 4), off_status = off_info + up((size_t)n_frames * nb);
    HostCtx *h = nullptr;
    rc = host_ctx(dev, stream, off_status + (size_t)n_frames * 4, &h);
    if (rc) return rc;
    float *llr_d = (float *)h->dbuf;
    uint8_t *info_d = (uint8_t *)h->dbuf + off_info;
    int32_t *status_d = (int32_t *)((char *)h->dbuf + off_status);
    int k = n_frames / kHostMinChunk;
    k = k < 1 ? 1 : (k > kHostChunks ? kHostChunks : k);
    const int per = (n_frames + k - 1) / k;
    CU(cudaEventRecord(h->ev_start, (cudaStream_t)stream));
    CU(cudaStreamWaitEvent(h->copy, h->ev_start, 0));
    CU(cudaStreamWaitEvent(h->comp[0], h->ev_start, 0));
    CU(cudaStreamWaitEvent(h->comp[1], h->ev_start, 0));
    for (int i = 0; i < k; i++) {
        const size_t f0 = (size_t)i * per, m = std::min((size_t)per, (size_t)n_frames - f0);
        CU(cudaMemcpyAsync(llr_d + f0 * row, llr_host + f0 * row, m * row * 4, cudaMemcpyHostToDevice, h->copy));
        CU(cudaEventRecord(h->ev_in[i], h->copy));
    }
    for (int i = 0; i < k; i++) {
        const size_t f0 = (size_t)i * per, m = std::min((size_t)per, (size_t)n_frames - f0);
        cudaStream_t s = h->comp[i & 1];
        CU(cudaStreamWaitEvent(s, h->ev_in[i], 0));
        rc = pscl_decode(c, llr_d + f0 * row, (int)m, L, algo, pr, quant, info_d + f0 * nb, status_d + f0, nullptr,
                         (void *)s);
        if (rc) {
            // a later chunk could not be enqueued (a device error): later
            // work on `stream` still waits for what was, so the caller's
            // buffers stay in use until it is done
            for (int j = 0; j < 2; j++) {
                cudaEventRecord(h->ev_done[j], h->comp[j]);
                cudaStreamWaitEvent((cudaStream_t)stream, h->ev_done[j], 0);
            }
            cudaEventRecord(h->ev_in[0], h->copy);
            cudaStreamWaitEvent((cudaStream_t)stream, h->ev_in[0], 0);
            return rc;
        }
        CU(cudaMemcpyAsync(info_host + f0 * nb, info_d + f0 * nb, m * nb, cudaMemcpyDeviceToHost, s));
        CU(cudaMemcpyAsync(status_host + f0, status_d + f0, m * 4, cudaMemcpyDeviceToHost, s));
    }
    for (int j = 0; j < 2; j++) {
        CU(cudaEventRecord(h->ev_done[j], h->comp[j]));
        CU(cudaStreamWaitEvent((cudaStream_t)stream, h->ev_done[j], 0));
    }
    return PSCL_OK;
}

extern "C" int pscl_decode_ws(pscl_code c, const float *llr, int n_frames, int L, pscl_algo algo,
                              const pscl_pruning *pr, pscl_quant quant, uint8_t *info_out, int32_t *status_out,
                              float *pm_out, void *workspace, size_t workspace_bytes, void *stream)
{
    Plan pl;
    int rc = make_plan(c, n_frames, L, algo, pr, quant, &pl);
    if (rc) return rc;
    return run_decode(c, llr, n_frames, L, algo, pr, quant, info_out, status_out, pm_out, workspace,
                      workspace_bytes, (cudaStream_t)stream, pl);
}

extern "C" int pscl_encode(pscl_code c, const uint8_t *info, int n_frames, uint8_t *x_out, void *stream)
{
    if (!c) return fail(PSCL_EINVAL, "code is NULL");
    if (n_frames < 0) return fail(PSCL_EINVAL, "n_frames=%d", n_frames);
    if (n_frames == 0) return PSCL_OK;
    if (!info || !x_out) return fail(PSCL_EINVAL, "info and x_out are required");
    EncParams p;
    p.code = c->dc;
    p.info = info;
    p.x = x_out;
    p.n_frames = n_frames;
    cudaError_t e = launch_encode(p, (cudaStream_t)stream);
    if (e != cudaSuccess) return fail(PSCL_ECUDA, "encode launch: %s", cudaGetErrorString(e));
    return PSCL_OK;
}

// ---------------------------------------------------------------------------
// diagnostics used by the tests and the benchmark (not part of the paper's
// method): kernel launches of the last decode call, the debug error word of
// the library workspace (bounds-checked builds), and the tuning knob.
extern "C" int pscl_debug_last_launches(void) { return g_last_launches; }

extern "C" int pscl_debug_error_word(uint32_t *out)
{
    int dev;
    CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    *out = 0;
    for (auto &kv : g_ws) {
        if (kv.first.first != dev || !kv.second.first) continue;
        uint32_t w = 0;
        CU(cudaMemcpy(&w, kv.second.first, 4, cudaMemcpyDeviceToHost));
        *out |= w;
    }
    return PSCL_OK;
}

extern "C" int pscl_set_tuning(int target_warps_per_sm)
{
    if (target_warps_per_sm < 1 || target_warps_per_sm > 64) return fail(PSCL_EINVAL, "target warps per SM out of range");
    g_target_warps_per_sm = target_warps_per_sm;
    return PSCL_OK;
}

extern "C" int pscl_set_sc_kernel(int enable)
{
    g_sc_kernel = enable != 0;
    return PSCL_OK;
}

extern "C" int pscl_set_fusion(int max_leaves)
{
    if (max_leaves != 0 && max_leaves != 1 && max_leaves != 2 && max_leaves != 4 && max_leaves != 8)
        return fail(PSCL_EINVAL, "fusion size %d: must be 1, 2, 4 or 8 (0 = by format)", max_leaves);
    g_fuse_max = max_leaves;
    return PSCL_OK;
}


extern "C" int pscl_debug_step_cycles(uint64_t *out, int reset)
{
#ifdef PSCL_OPPROF
    if (!out) return fail(PSCL_EINVAL, "out is NULL");
    unsigned long long *p = prof_buffer();
    if (!p) return fail(PSCL_ECUDA, "profile counters unavailable");
    CU(cudaDeviceSynchronize());
    CU(cudaMemcpy(out, p, 32 * sizeof(unsigned long long), cudaMemcpyDeviceToHost));
    if (reset) CU(cudaMemset(p, 0, 32 * sizeof(unsigned long long)));
    return PSCL_OK;
#else
    (void)out;
    (void)reset;
    return fail(PSCL_EUNSUPPORTED, "not a step-profiling build");
#endif
}

extern "C" int pscl_debug_checked(void)
{
#ifdef PSCL_CHECKED
    return 1;
#else
    return 0;
#endif
}

// ---------------------------------------------------------------------------
// Decoding without any allocation.
//
// Some callers cannot allocate device memory at decode time: code running
// where cudaMalloc is forbidden or would stall (a real-time receive loop that
// must not synchronise the device, a host process whose memory is handed out
// by another allocator, or work that is set up once and then only launched).
// pscl_decode_static serves them: its scratch is the file-scope device array
// below, of PSCL_STATIC_SCRATCH_BYTES bytes, which every GPU that loads this
// library holds until the process exits.  Its device address is looked up
// once per device with cudaGetSymbolAddress (a host-side name of the array is
// not a device address).
#define PSCL_STATIC_SCRATCH_BYTES (32u << 20)
static __device__ __align__(256) unsigned char g_static_scratch[PSCL_STATIC_SCRATCH_BYTES];
static std::map<int, void *> g_static_ptr;

static int static_scratch(void **out)
{
    int dev;
    CU(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_static_ptr.find(dev);
    if (it == g_static_ptr.end()) {
        void *ptr = nullptr;
        CU(cudaGetSymbolAddress(&ptr, g_static_scratch));
        it = g_static_ptr.emplace(dev, ptr).first;
    }
    *out = it->second;
    return PSCL_OK;
}

extern "C" int pscl_decode_static(pscl_code c, const float *llr, int n_frames, int L, pscl_algo algo,
                                  const pscl_pruning *pr, pscl_quant quant, uint8_t *info_out,
                                  int32_t *status_out, float *pm_out, void *stream)
{
    Plan pl;
    int rc = make_plan(c, n_frames, L, algo, pr, quant, &pl, false);
    if (rc) return rc;
    void *ws;
    rc = static_scratch(&ws);
    if (rc) return rc;
    // fit the resident warps to the array: frames beyond them are handled by
    // the kernel's task loop, so only the per-warp slice and the adaptive
    // frame lists bound what can be decoded
    const size_t fixed = 256 + pl.list_bytes;
    const size_t per_warp = pl.total_warps ? pl.gmem_scratch / (size_t)pl.total_warps : 0;
    const int wpb = pl.warps_per_block;
    if (fixed + (size_t)wpb * per_warp > PSCL_STATIC_SCRATCH_BYTES)
        return fail(PSCL_EINVAL,
                    "pscl_decode_static: needs %zu bytes of scratch (%zu for frame lists, %zu per warp x %d) "
                    "but its static scratch holds %u bytes",
                    fixed + (size_t)wpb * per_warp, pl.list_bytes, per_warp, wpb, PSCL_STATIC_SCRATCH_BYTES);
    if (per_warp > 0) {
        size_t fit = (PSCL_STATIC_SCRATCH_BYTES - fixed) / per_warp;
        if (fit < (size_t)pl.total_warps) {
            pl.total_warps = (int)(fit / wpb) * wpb;
            pl.grid = pl.total_warps / wpb;
            pl.gmem_scratch = per_warp * (size_t)pl.total_warps;
            pl.total_ws = fixed + pl.gmem_scratch;
        }
    }
    // the debug word and the list counters start at zero on every call
    CU(cudaMemsetAsync(ws, 0, 256, (cudaStream_t)stream));
    return run_decode(c, llr, n_frames, L, algo, pr, quant, info_out, status_out, pm_out, ws,
                      PSCL_STATIC_SCRATCH_BYTES, (cudaStream_t)stream, pl);
}

// ---------------------------------------------------------------------------
// Uneven batches: many work items (codes, list sizes, number formats) in one
// persistent launch per number format.  The plan owns a device item table, a
// task list sorted longest-first, a task counter and the warps' scratch, so
// running it allocates nothing and can be captured in a CUDA graph.
struct BatchGroup {
    int quant = 0;
    bool nodes = false;
    int kv = KV_PLAIN;
    int n_tasks = 0;
    int grid = 0;
    int total_warps = 0;
    size_t smem_block = 0;
    uint32_t smem_per_warp = 0, gmem_per_warp = 0;
    int2 *d_tasks = nullptr;
    int *d_ctr = nullptr;
    char *d_gmem = nullptr;
    std::vector<int> items;          // item indices of this group
    std::vector<std::vector<int2>> item_tasks;
};

struct pscl_batch_s {
    int dev = -1;
    std::vector<pscl_work_item> wi;
    std::vector<Item> h_items;
    Item *d_items = nullptr;
    uint32_t *d_err = nullptr;
    std::vector<BatchGroup> groups;
    std::vector<void *> allocs;
};

static void batch_free(pscl_batch b)
{
    for (void *p : b->allocs) lib_free(p);
    delete b;
}

extern "C" int pscl_batch_create(const pscl_work_item *items, int n_items, pscl_batch *out)
{
    if (!out) return fail(PSCL_EINVAL, "out is NULL");
    *out = nullptr;
    if (!items || n_items < 1) return fail(PSCL_EINVAL, "no work items");
    DevProps dp;
    int rc = get_props(&dp);
    if (rc) return rc;
    int dev;
    CU(cudaGetDevice(&dev));
    pscl_batch b = new pscl_batch_s();
    b->dev = dev;
    b->wi.assign(items, items + n_items);
    b->h_items.resize((size_t)n_items);
    std::vector<Program> progs((size_t)n_items);
    for (int i = 0; i < n_items; i++) {
        const pscl_work_item &w = items[i];
        if (!w.code || w.code->dev != dev) { batch_free(b); return fail(PSCL_EINVAL, "item %d: bad code", i); }
        if (w.algo != PSCL_SC && w.algo != PSCL_CASCL) {
            batch_free(b);
            return fail(PSCL_EUNSUPPORTED, "item %d: batches take SC or CASCL items", i);
        }
        if (w.L != 1 && w.L != 2 && w.L != 4 && w.L != 8 && w.L != 16 && w.L != 32) {
            batch_free(b);
            return fail(PSCL_EINVAL, "item %d: L=%d", i, w.L);
        }
        if (w.quant < PSCL_F32 || w.quant > PSCL_I8 || w.n_frames < 0) {
            batch_free(b);
            return fail(PSCL_EINVAL, "item %d: bad quantisation or frame count", i);
        }
        int wps_i, fuse_i;
        tuning_for(w.code, w.algo == PSCL_SC ? 1 : w.L, (int)w.quant, w.pruning, &wps_i, &fuse_i);
        rc = get_program(w.code, w.pruning, fuse_i, w.quant != PSCL_F32, &progs[(size_t)i]);
        if (rc) { batch_free(b); return rc; }
    }
    void *p;
    cudaError_t e = cudaMalloc(&p, 256);
    if (e != cudaSuccess) { batch_free(b); return fail(PSCL_ENOMEM, "batch: %s", cudaGetErrorString(e)); }
    b->allocs.push_back(p);
    b->d_err = (uint32_t *)p;
    cudaMemset(p, 0, 256);
    const size_t budget = slice_budget(dp, g_target_warps_per_sm);
    for (int q = PSCL_F32; q <= PSCL_I8; q++) {
        BatchGroup g;
        g.quant = q;
        std::vector<std::pair<double, int2>> tasks;
        for (int i = 0; i < n_items; i++) {
            const pscl_work_item &w = items[i];
            if ((int)w.quant != q || w.n_frames == 0) continue;
            const int L = w.algo == PSCL_SC ? 1 : w.L;
            Item &it = b->h_items[(size_t)i];
            memset(&it, 0, sizeof(it));
            it.code = w.code->dc;
            it.ops = progs[(size_t)i].d_ops;
            it.n_ops = progs[(size_t)i].n_ops;
            it.root_special = progs[(size_t)i].root_special;
            make_layout(w.code, progs[(size_t)i], L, q, budget, &it.lay);
            it.llr_off = w.llr_offset;
            it.info_off = w.info_offset;
            it.status_off = (int)w.status_offset;
            it.n_frames = w.n_frames;
            it.L = L;
            it.L_out = L;
            it.stage_L = L;
            it.err = b->d_err;
            if (progs[(size_t)i].has_nodes) g.nodes = true;
            if (it.lay.smem_per_warp > g.smem_per_warp) g.smem_per_warp = it.lay.smem_per_warp;
            if (it.lay.gmem_per_warp > g.gmem_per_warp) g.gmem_per_warp = it.lay.gmem_per_warp;
            g.items.push_back(i);
            // a task decodes 32/L frames of one item; cost ~ N log N grows
            // with the list size through the selections
            const int fpw = 32 / L;
            const double cost = (double)w.code->N * (double)(w.code->n) * (1.0 + 0.25 * __builtin_ctz((unsigned)L));
            for (int f = 0; f < w.n_frames; f += fpw) tasks.push_back({cost, make_int2(i, f)});
        }
        if (tasks.empty()) continue;
        std::stable_sort(tasks.begin(), tasks.end(),
                         [](const std::pair<double, int2> &a, const std::pair<double, int2> &b2) { return a.first > b2.first; });
        std::vector<int2> h_tasks(tasks.size());
        for (size_t k = 0; k < tasks.size(); k++) h_tasks[k] = tasks[k].second;
        g.n_tasks = (int)h_tasks.size();
        g.smem_block = (size_t)g.smem_per_warp * kWarpsPerBlock;
        int bps = 0;
        g.kv = kernel_variant(g.nodes, g_target_warps_per_sm);
        e = scl_func_attrs(q, g.kv, g.smem_block, 32 * kWarpsPerBlock, &bps);
        if (e != cudaSuccess || bps < 1) {
            batch_free(b);
            return fail(PSCL_EUNSUPPORTED, "batch: no block fits (%zu bytes of shared memory)", g.smem_block);
        }
        const int max_warps = dp.sms * bps * kWarpsPerBlock;
        const int tw = g.n_tasks < max_warps ? g.n_tasks : max_warps;
        g.grid = (tw + kWarpsPerBlock - 1) / kWarpsPerBlock;
        g.total_warps = g.grid * kWarpsPerBlock;
        e = cudaMalloc(&p, sizeof(int2) * h_tasks.size());
        if (e == cudaSuccess) {
            b->allocs.push_back(p);
            g.d_tasks = (int2 *)p;
            e = cudaMemcpy(p, h_tasks.data(), sizeof(int2) * h_tasks.size(), cudaMemcpyHostToDevice);
        }
        if (e == cudaSuccess) {
            e = cudaMalloc(&p, 256 + (size_t)g.gmem_per_warp * (size_t)g.total_warps);
            if (e == cudaSuccess) {
                b->allocs.push_back(p);
                g.d_ctr = (int *)p;
                g.d_gmem = (char *)p + 256;
            }
        }
        if (e != cudaSuccess) {
            batch_free(b);
            return fail(PSCL_ENOMEM, "batch: %s", cudaGetErrorString(e));
        }
        // per-item task lists for the one-launch-per-item form
        g.item_tasks.resize(g.items.size());
        b->groups.push_back(g);
    }
    e = cudaMalloc(&p, sizeof(Item) * (size_t)n_items);
    if (e == cudaSuccess) {
        b->allocs.push_back(p);
        b->d_items = (Item *)p;
        e = cudaMemcpy(p, b->h_items.data(), sizeof(Item) * (size_t)n_items, cudaMemcpyHostToDevice);
    }
    if (e != cudaSuccess) {
        batch_free(b);
        return fail(PSCL_ENOMEM, "batch: %s", cudaGetErrorString(e));
    }
    *out = b;
    return PSCL_OK;
}

extern "C" int pscl_batch_destroy(pscl_batch b)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    batch_free(b);
    return PSCL_OK;
}

extern "C" int pscl_batch_run(pscl_batch b, const float *llr_pool, uint8_t *info_pool, int32_t *status_pool,
                              void *stream)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    if (!llr_pool || !info_pool || !status_pool) return fail(PSCL_EINVAL, "pools are required");
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    for (const BatchGroup &g : b->groups) {
        KParams kp;
        memset(&kp, 0, sizeof(kp));
        kp.items = b->d_items;
        kp.tasks = g.d_tasks;
        kp.n_tasks = g.n_tasks;
        kp.task_ctr = g.d_ctr;
        kp.gmem = g.d_gmem;
        kp.gmem_per_warp = g.gmem_per_warp;
        kp.smem_per_warp = g.smem_per_warp;
        kp.total_warps = g.total_warps;
        kp.llr_pool = llr_pool;
        kp.info_pool = info_pool;
        kp.status_pool = status_pool;
        CU(cudaMemsetAsync(g.d_ctr, 0, sizeof(int), s));
        cudaError_t e = launch_stage(g.quant, g.kv, kp, g.grid, g.smem_block, s);
        if (e != cudaSuccess) return fail(PSCL_ECUDA, "batch launch: %s", cudaGetErrorString(e));
        launches++;
    }
    g_last_launches = launches;
    return PSCL_OK;
}

// The same batch decoded one launch per work item (no overlap between items,
// no task counter): the plain form the persistent launch is measured against.
extern "C" int pscl_batch_run_plain(pscl_batch b, const float *llr_pool, uint8_t *info_pool,
                                    int32_t *status_pool, void *stream)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    if (!llr_pool || !info_pool || !status_pool) return fail(PSCL_EINVAL, "pools are required");
    cudaStream_t s = (cudaStream_t)stream;
    int launches = 0;
    for (const BatchGroup &g : b->groups) {
        for (int i : g.items) {
            const pscl_work_item &w = b->wi[(size_t)i];
            KParams kp;
            memset(&kp, 0, sizeof(kp));
            kp.single = b->h_items[(size_t)i];
            kp.single.llr = llr_pool + w.llr_offset;
            kp.single.info_out = info_pool + w.info_offset;
            kp.single.status_out = status_pool + w.status_offset;
            kp.single.pm_out = nullptr;
            const int fpw = 32 / kp.single.L;
            const int tasks = (w.n_frames + fpw - 1) / fpw;
            const int tw = tasks < g.total_warps ? tasks : g.total_warps;
            const int grid = (tw + kWarpsPerBlock - 1) / kWarpsPerBlock;
            kp.gmem = g.d_gmem;
            kp.gmem_per_warp = g.gmem_per_warp;
            kp.smem_per_warp = kp.single.lay.smem_per_warp;
            kp.total_warps = grid * kWarpsPerBlock;
            cudaError_t e = launch_stage(g.quant, g.kv, kp, grid, (size_t)kp.smem_per_warp * kWarpsPerBlock, s);
            if (e != cudaSuccess) return fail(PSCL_ECUDA, "plain launch: %s", cudaGetErrorString(e));
            launches++;
        }
    }
    g_last_launches = launches;
    return PSCL_OK;
}

extern "C" int pscl_batch_info(pscl_batch b, int *n_launches, int *n_tasks, size_t *scratch_bytes)
{
    if (!b) return fail(PSCL_EINVAL, "batch is NULL");
    int t = 0;
    size_t bytes = 0;
    for (const BatchGroup &g : b->groups) {
        t += g.n_tasks;
        bytes += (size_t)g.gmem_per_warp * (size_t)g.total_warps;
    }
    if (n_launches) *n_launches = (int)b->groups.size();
    if (n_tasks) *n_tasks = t;
    if (scratch_bytes) *scratch_bytes = bytes;
    return PSCL_OK;
}

// ---------------------------------------------------------------------------
// Serving loop: host side (device side in server.cu).
static uint64_t host_ns()
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (uint64_t)ts.tv_sec * 1000000000ull + (uint64_t)ts.tv_nsec;
}

struct SrvCtxInfo {
    size_t smem_per_warp = 0;     // shared-memory slice the context's layout needs
    size_t scratch_per_warp = 0;  // global scratch slice the context's layout needs
    size_t bytes_per_frame = 0;   // device bytes a frame of it holds while in flight
};

struct pscl_server_s {
    int dev = -1;
    bool nodes = false;
    int R = 0;
    int max_frames = 0;
    long long max_inflight = 0;
    long long hbm_budget = 0;     // 0 = no byte budget
    long long inflight_bytes = 0;
    std::vector<SrvCtxInfo> ctx_info;
    std::vector<long long> slot_bytes;
    int grid = 0, total_warps = 0;
    size_t smem_block = 0;
    std::vector<Item> h_items;
    std::vector<pscl_code> codes;
    Item *d_items = nullptr;
    SrvCtl *ctl = nullptr;      // mapped host memory (host view)
    SrvReq *ring = nullptr;
    SrvComp *comp = nullptr;
    char *d_mem = nullptr;      // device: counters, requests, claims, scratch
    cudaStream_t stream = nullptr;
    bool running = false;
    std::mutex mu;
    uint64_t next_ticket = 0;
    std::vector<uint64_t> slot_ticket;
    std::vector<char> slot_busy;
    std::vector<uint64_t> slot_submit_ns;
    std::vector<int> slot_frames;
    long long inflight = 0;
    uint64_t completed = 0;
};

static void server_free(pscl_server s)
{
    lib_free(s->d_items);
    lib_free(s->d_mem);
    lib_free(s->ctl, true);
    lib_free(s->ring, true);
    lib_free(s->comp, true);
    if (s->stream) cudaStreamDestroy(s->stream);
    delete s;
}

extern "C" int pscl_server_start(const pscl_server_cfg *cfg, pscl_server *out)
{
    if (!cfg || !out) return fail(PSCL_EINVAL, "cfg and out are required");
    *out = nullptr;
    const int R = cfg->ring_slots;
    if (R < 2 || R > 65536 || (R & (R - 1))) return fail(PSCL_EINVAL, "ring_slots=%d: a power of two in [2, 65536]", R);
    if (cfg->n_contexts < 1 || !cfg->contexts) return fail(PSCL_EINVAL, "no decoding contexts");
    if (cfg->max_frames_per_request < 1) return fail(PSCL_EINVAL, "max_frames_per_request < 1");
    if (cfg->idle_timeout_ms < 1) return fail(PSCL_EINVAL, "idle_timeout_ms < 1");
    if (cfg->hbm_budget_bytes < 0) return fail(PSCL_EINVAL, "hbm_budget_bytes < 0");
    DevProps dp;
    int rc = get_props(&dp);
    if (rc) return rc;
    pscl_server s = new pscl_server_s();
    CU(cudaGetDevice(&s->dev));
    s->R = R;
    s->max_frames = cfg->max_frames_per_request;
    s->max_inflight = cfg->max_inflight_frames > 0 ? cfg->max_inflight_frames : (long long)R * cfg->max_frames_per_request;
    s->hbm_budget = cfg->hbm_budget_bytes;
    // the serving kernel keeps 4 blocks of 4 warps per SM (its registers):
    // slices are sized for at most that many
    const size_t budget = slice_budget(dp, g_target_warps_per_sm < 16 ? g_target_warps_per_sm : 16);
    uint32_t smem_pw = 0, gmem_pw = 0;
    unsigned quant_mask = 0;
    s->h_items.resize((size_t)cfg->n_contexts);
    s->ctx_info.resize((size_t)cfg->n_contexts);
    for (int i = 0; i < cfg->n_contexts; i++) {
        const pscl_context &cx = cfg->contexts[i];
        if (!cx.code || cx.code->dev != s->dev) { server_free(s); return fail(PSCL_EINVAL, "context %d: bad code", i); }
        if (cx.L != 1 && cx.L != 2 && cx.L != 4 && cx.L != 8 && cx.L != 16 && cx.L != 32) {
            server_free(s);
            return fail(PSCL_EINVAL, "context %d: L=%d", i, cx.L);
        }
        if (cx.quant < PSCL_F32 || cx.quant > PSCL_I8) {
            server_free(s);
            return fail(PSCL_EINVAL, "context %d: unknown quantisation %d", i, (int)cx.quant);
        }
        const int q = (int)cx.quant;
        quant_mask |= 1u << q;
        int wps, fuse;
        tuning_for(cx.code, cx.L, q, cx.pruning, &wps, &fuse);
        Program pg;
        rc = get_program(cx.code, cx.pruning, fuse, q != PSCL_F32, &pg);
        if (rc) { server_free(s); return rc; }
        if (pg.has_nodes) s->nodes = true;
        Item &it = s->h_items[(size_t)i];
        memset(&it, 0, sizeof(it));
        it.code = cx.code->dc;
        it.ops = pg.d_ops;
        it.n_ops = pg.n_ops;
        it.root_special = pg.root_special;
        make_layout(cx.code, pg, cx.L, q, budget, &it.lay);
        it.L = cx.L;
        it.L_out = cx.L;
        it.llr_cg = 1;
        it.stage_L = cx.L;
        it.quant = q;
        if (it.lay.smem_per_warp > smem_pw) smem_pw = it.lay.smem_per_warp;
        if (it.lay.gmem_per_warp > gmem_pw) gmem_pw = it.lay.gmem_per_warp;
        // device footprint of one frame in flight: its LLR row, its output
        // row and status word, and its share of a warp's scratch slice
        SrvCtxInfo &ci = s->ctx_info[(size_t)i];
        ci.smem_per_warp = it.lay.smem_per_warp;
        ci.scratch_per_warp = it.lay.gmem_per_warp;
        ci.bytes_per_frame = (size_t)(cx.code->N - cx.code->P) * 4 + (size_t)((cx.code->kinfo + 7) / 8) + 4 +
                             (size_t)it.lay.gmem_per_warp * (size_t)cx.L / 32;
        if (s->hbm_budget > 0 && (long long)ci.bytes_per_frame > s->hbm_budget) {
            server_free(s);
            return fail(PSCL_EINVAL, "context %d: one frame needs %zu bytes, more than the HBM budget %lld", i,
                        ci.bytes_per_frame, s->hbm_budget);
        }
        s->codes.push_back(cx.code);
    }
    s->smem_block = (size_t)smem_pw * kWarpsPerBlock;
    int bps = 0;
    cudaError_t e = server_attrs(s->nodes, s->smem_block, &bps);
    if (e != cudaSuccess || bps < 1) {
        server_free(s);
        return fail(PSCL_EUNSUPPORTED, "server: no block fits (%zu bytes of shared memory)", s->smem_block);
    }
    int warps = dp.sms * bps * kWarpsPerBlock;
    if (cfg->max_warps > 0 && cfg->max_warps < warps) warps = cfg->max_warps / kWarpsPerBlock * kWarpsPerBlock;
    if (warps < kWarpsPerBlock) warps = kWarpsPerBlock;
    s->grid = warps / kWarpsPerBlock;
    s->total_warps = s->grid * kWarpsPerBlock;
    // device memory: counters | open requests | claims | done | scratch
    const size_t off_dreq = 256, off_claim = off_dreq + sizeof(SrvDReq) * (size_t)R,
                 off_done = off_claim + 8 * (size_t)R, off_gmem = (off_done + 4 * (size_t)R + 255) & ~(size_t)255,
                 total = off_gmem + (size_t)gmem_pw * (size_t)s->total_warps;
    e = cudaMalloc(&s->d_mem, total);
    if (e == cudaSuccess) e = cudaMemset(s->d_mem, 0, off_gmem);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_items, sizeof(Item) * s->h_items.size());
    if (e == cudaSuccess)
        e = cudaMemcpy(s->d_items, s->h_items.data(), sizeof(Item) * s->h_items.size(), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->ctl, sizeof(SrvCtl), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->ring, sizeof(SrvReq) * (size_t)R, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&s->comp, sizeof(SrvComp) * (size_t)R, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        server_free(s);
        return fail(e == cudaErrorMemoryAllocation ? PSCL_ENOMEM : PSCL_ECUDA, "server: %s", cudaGetErrorString(e));
    }
    memset(s->ctl, 0, sizeof(SrvCtl));
    memset(s->ring, 0, sizeof(SrvReq) * (size_t)R);
    memset(s->comp, 0, sizeof(SrvComp) * (size_t)R);
    s->slot_ticket.assign((size_t)R, 0);
    s->slot_busy.assign((size_t)R, 0);
    s->slot_submit_ns.assign((size_t)R, 0);
    s->slot_frames.assign((size_t)R, 0);
    s->slot_bytes.assign((size_t)R, 0);
    SrvParams P;
    memset(&P, 0, sizeof(P));
    P.K.items = s->d_items;
    P.K.gmem = s->d_mem + off_gmem;
    P.K.gmem_per_warp = gmem_pw;
    P.K.smem_per_warp = smem_pw;
    P.K.total_warps = s->total_warps;
    P.n_ctx = cfg->n_contexts;
    P.quant_mask = quant_mask;
    void *dp_ctl, *dp_ring, *dp_comp;
    cudaHostGetDevicePointer(&dp_ctl, s->ctl, 0);
    cudaHostGetDevicePointer(&dp_ring, s->ring, 0);
    cudaHostGetDevicePointer(&dp_comp, s->comp, 0);
    P.ctl = (SrvCtl *)dp_ctl;
    P.ring = (SrvReq *)dp_ring;
    P.comp = (SrvComp *)dp_comp;
    P.dev = (SrvDev *)s->d_mem;
    P.dreq = (SrvDReq *)(s->d_mem + off_dreq);
    P.claim = (unsigned long long *)(s->d_mem + off_claim);
    P.done = (uint32_t *)(s->d_mem + off_done);
    P.R = R;
    P.idle_ns = (unsigned long long)cfg->idle_timeout_ms * 1000000ull;
    e = server_launch(s->nodes, P, s->grid, s->smem_block, s->stream);
    if (e != cudaSuccess) {
        server_free(s);
        return fail(PSCL_ECUDA, "server launch: %s", cudaGetErrorString(e));
    }
    server_started(s->dev);
    s->running = true;
    *out = s;
    return PSCL_OK;
}

extern "C" int pscl_server_submit(pscl_server s, const pscl_request *req, uint64_t *ticket)
{
    if (!s || !req) return fail(PSCL_EINVAL, "server and request are required");
    if (req->context < 0 || req->context >= (int)s->h_items.size())
        return fail(PSCL_EINVAL, "request context %d out of range", req->context);
    if (req->n_frames < 1 || req->n_frames > s->max_frames)
        return fail(PSCL_EINVAL, "request of %d frames (1..%d)", req->n_frames, s->max_frames);
    if (!req->llr || !req->info_out || !req->status_out) return fail(PSCL_EINVAL, "request buffers are required");
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->running && *(volatile int32_t *)&s->ctl->exit_status != 0 && cudaStreamQuery(s->stream) == cudaSuccess)
        s->running = false;  // the kernel left on its idle budget
    if (!s->running) return fail(PSCL_EINVAL, "server is stopped");
    const uint64_t t = s->next_ticket;
    const int slot = (int)(t & (uint64_t)(s->R - 1));
    const long long bytes = (long long)s->ctx_info[(size_t)req->context].bytes_per_frame * req->n_frames;
    if (s->hbm_budget > 0 && bytes > s->hbm_budget)
        return fail(PSCL_EINVAL, "request of %lld device bytes exceeds the whole HBM budget %lld", bytes, s->hbm_budget);
    if (s->slot_busy[(size_t)slot] || s->inflight + req->n_frames > s->max_inflight ||
        (s->hbm_budget > 0 && s->inflight_bytes + bytes > s->hbm_budget))
        return fail(PSCL_EAGAIN, "server full: %lld frames (%lld bytes) in flight", s->inflight, s->inflight_bytes);
    SrvReq &r = s->ring[slot];
    r.ctx = req->context;
    r.n = req->n_frames;
    r.llr = req->llr;
    r.info = req->info_out;
    r.status = req->status_out;
    s->slot_ticket[(size_t)slot] = t;
    s->slot_busy[(size_t)slot] = 1;
    s->slot_submit_ns[(size_t)slot] = host_ns();
    s->slot_frames[(size_t)slot] = req->n_frames;
    s->slot_bytes[(size_t)slot] = bytes;
    s->inflight += req->n_frames;
    s->inflight_bytes += bytes;
    s->next_ticket = t + 1;
    std::atomic_thread_fence(std::memory_order_seq_cst);
    *(volatile uint32_t *)&s->ctl->tail = (uint32_t)(t + 1);
    std::atomic_thread_fence(std::memory_order_seq_cst);
    if (ticket) *ticket = t;
    return PSCL_OK;
}

extern "C" int pscl_server_poll(pscl_server s, pscl_completion *out, int max, int *n_out)
{
    if (!s || !n_out || (max > 0 && !out)) return fail(PSCL_EINVAL, "bad arguments");
    std::lock_guard<std::mutex> lk(s->mu);
    // once the kernel has left (idle budget or stop), requests it never
    // finished are reported as failed instead of staying outstanding
    const int xs = *(volatile int32_t *)&s->ctl->exit_status;
    const bool gone = xs != 0 && cudaStreamQuery(s->stream) == cudaSuccess;
    if (gone) s->running = false;
    int n = 0;
    for (int slot = 0; slot < s->R && n < max; slot++) {
        if (!s->slot_busy[(size_t)slot]) continue;
        volatile SrvComp *c = s->comp + slot;
        const uint64_t t = s->slot_ticket[(size_t)slot];
        const bool done = c->seq == (uint32_t)(t + 1);
        if (!done && !gone) continue;
        std::atomic_thread_fence(std::memory_order_acquire);
        pscl_completion &o = out[n++];
        o.ticket = t;
        o.status = done ? c->status : xs;
        o.n_frames = s->slot_frames[(size_t)slot];
        o.t_submit_ns = s->slot_submit_ns[(size_t)slot];
        o.t_done_ns = host_ns();
        o.device_ns = done ? c->t_end - c->t_open : 0;
        s->slot_busy[(size_t)slot] = 0;
        s->inflight -= o.n_frames;
        s->inflight_bytes -= s->slot_bytes[(size_t)slot];
        s->completed++;
    }
    *n_out = n;
    return PSCL_OK;
}

extern "C" int pscl_server_context_info(pscl_server s, int context, size_t *smem_per_warp, size_t *scratch_per_warp,
                                        size_t *bytes_per_frame)
{
    if (!s) return fail(PSCL_EINVAL, "server is NULL");
    if (context < 0 || context >= (int)s->ctx_info.size()) return fail(PSCL_EINVAL, "context %d out of range", context);
    const SrvCtxInfo &ci = s->ctx_info[(size_t)context];
    if (smem_per_warp) *smem_per_warp = ci.smem_per_warp;
    if (scratch_per_warp) *scratch_per_warp = ci.scratch_per_warp;
    if (bytes_per_frame) *bytes_per_frame = ci.bytes_per_frame;
    return PSCL_OK;
}

extern "C" int pscl_debug_server_exit(pscl_server s, int *warp, long long *idle_ns, unsigned long long *budget_ns,
                                      uint32_t *tickets)
{
    if (!s) return fail(PSCL_EINVAL, "server is NULL");
    volatile SrvCtl *c = s->ctl;
    if (warp) *warp = (int)c->exit_warp;
    if (idle_ns) *idle_ns = c->exit_idle_ns;
    if (budget_ns) *budget_ns = c->exit_budget_ns;
    if (tickets) {
        tickets[0] = c->exit_opened;
        tickets[1] = c->exit_head;
        tickets[2] = c->exit_opening;
        tickets[3] = c->exit_tail;
    }
    return PSCL_OK;
}

extern "C" int pscl_debug_server_slots(pscl_server s, uint64_t *claim, uint32_t *done, int32_t *nframes,
                                       uint64_t *tickets)
{
    if (!s) return fail(PSCL_EINVAL, "server is NULL");
    if (cudaStreamQuery(s->stream) != cudaSuccess) return fail(PSCL_EINVAL, "the serving kernel is still running");
    const size_t R = (size_t)s->R;
    const size_t off_dreq = 256, off_claim = off_dreq + sizeof(SrvDReq) * R, off_done = off_claim + 8 * R;
    std::vector<SrvDReq> dr(R);
    CU(cudaMemcpy(claim, s->d_mem + off_claim, 8 * R, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(done, s->d_mem + off_done, 4 * R, cudaMemcpyDeviceToHost));
    CU(cudaMemcpy(dr.data(), s->d_mem + off_dreq, sizeof(SrvDReq) * R, cudaMemcpyDeviceToHost));
    for (size_t k = 0; k < R; k++) {
        nframes[k] = dr[k].n;
        tickets[k] = s->slot_busy[k] ? s->slot_ticket[k] : ~0ull;
    }
    return PSCL_OK;
}

extern "C" int pscl_server_status(pscl_server s, int *running, int *device_status, uint64_t *completed,
                                  long long *frames_in_flight)
{
    if (!s) return fail(PSCL_EINVAL, "server is NULL");
    std::lock_guard<std::mutex> lk(s->mu);
    const bool alive = cudaStreamQuery(s->stream) == cudaErrorNotReady;
    if (running) *running = alive ? 1 : 0;
    if (device_status) *device_status = s->ctl->exit_status;
    if (completed) *completed = s->completed;
    if (frames_in_flight) *frames_in_flight = s->inflight;
    return PSCL_OK;
}

extern "C" int pscl_server_stop(pscl_server s, int timeout_ms)
{
    if (!s) return fail(PSCL_EINVAL, "server is NULL");
    {
        std::lock_guard<std::mutex> lk(s->mu);
        s->running = false;
        std::atomic_thread_fence(std::memory_order_seq_cst);
        *(volatile uint32_t *)&s->ctl->abort = 1u;
        std::atomic_thread_fence(std::memory_order_seq_cst);
    }
    const uint64_t t0 = host_ns();
    for (;;) {
        cudaError_t q = cudaStreamQuery(s->stream);
        if (q == cudaSuccess) break;
        if (q != cudaErrorNotReady) return fail(PSCL_ECUDA, "server stream: %s", cudaGetErrorString(q));
        if (host_ns() - t0 > (uint64_t)timeout_ms * 1000000ull)
            return fail(PSCL_ETIMEDOUT, "the serving loop did not stop within %d ms (resources kept)", timeout_ms);
        struct timespec ts = {0, 200000};
        nanosleep(&ts, nullptr);
    }
    const int dev = s->dev;
    server_free(s);
    server_stopped(dev);
    return PSCL_OK;
}
