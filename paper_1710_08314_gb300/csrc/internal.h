// internal.h -- structures shared by the host side of libpolarscl and its
// kernels.  Not part of the public ABI (see include/polarscl.h).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pscl {

constexpr int kMaxLog2N = 13;          // N <= 8192
constexpr int kMaxLayers = kMaxLog2N + 1;
// per-path slot tables hold layers 1..kTabLayers (layer 0, the channel
// LLRs, is shared by the paths of a frame): schedules deeper than that are
// refused (with register subtrees of 2 or more leaves, N = 8192 fits)
constexpr int kTabLayers = 12;

// One instruction of the node schedule a warp walks for a code (the
// pre-order traversal of Algorithm 1, with pruned nodes as single steps).
//   bits 0..3  opcode      bits 4..7  depth d      bits 8..10 node type
//   bit  11    side (0 = left child, 1 = right child or root)
//   bits 12..15 flip depth t   (OP_RSUB: bits 16..31 frozen-leaf mask)
enum Opcode : uint32_t {
    OP_F = 0,     // layer d+1 = f(layer d)               (left child LLRs)
    OP_G = 1,     // layer d+1 = g(layer d, beta_left)     (right child LLRs)
    OP_NODE = 2,  // leaf or pruned node at depth d
    OP_COMB = 3,  // right child at depth d done: parent beta = h(left, right)
    OP_RSUB = 4,  // unpruned subtree of 2..8 leaves at depth d, decoded in
                  //   registers; bits 16..31: frozen mask of its leaves
    OP_RSUB2 = 5, // unpruned subtree of 2H leaves (H = 2..8) at depth d: f,
                  //   left half in registers, g, right half in registers, h;
                  //   the node's LLRs are read twice from layer d and its
                  //   children's LLRs never reach memory; bits 16..31 as above;
                  //   t = 1 | parent side << 1: the node is a right child and
                  //   the parent's h step (OP_COMB) is folded in
    OP_RSUB4 = 6, // unpruned subtree of 16 leaves (H = 4) at depth d: four
                  //   register subtrees of H leaves, the node's LLRs read once
                  //   per quarter; fields as OP_RSUB2
};
enum NodeType : uint32_t { NT_R0 = 1, NT_R1 = 2, NT_REP = 3, NT_SPC = 4 };

__host__ __device__ inline uint32_t op_make(uint32_t code, uint32_t d, uint32_t type, uint32_t side,
                                            uint32_t t)
{
    return code | (d << 4) | (type << 8) | (side << 11) | (t << 12);
}
__host__ __device__ inline uint32_t op_code(uint32_t w) { return w & 15u; }
__host__ __device__ inline int op_depth(uint32_t w) { return (int)((w >> 4) & 15u); }
__host__ __device__ inline uint32_t op_type(uint32_t w) { return (w >> 8) & 7u; }
__host__ __device__ inline int op_side(uint32_t w) { return (int)((w >> 11) & 1u); }
__host__ __device__ inline int op_t(uint32_t w) { return (int)((w >> 12) & 15u); }

// Device-resident description of a code.
struct DevCode {
    int N, n, K, kinfo, crc_len, systematic, P;
    uint32_t poly32;            // crc_poly << (32 - crc_len)
    const int32_t *in_index;    // N: column of position i in an LLR row, -1 if punctured
    const uint16_t *A;          // K information positions, increasing
    const uint32_t *amask;      // max(1, N/32) words: bit set for positions in A
    const uint32_t *crc_lut;    // 256 entries, MSB-first table for the 32-bit-aligned CRC
    const uint32_t *syn;        // N/8 x 256: CRC syndrome contribution of codeword byte q with value v
    const uint8_t *ext;         // N/8 x 256: the info bits of codeword byte q with value v, packed LSB first
    const uint16_t *ext_pos;    // N/8 + 1: index of the first info bit of codeword byte q in u_A
};

// Per-warp memory map.  Offsets are bytes inside the warp's shared-memory
// slice (bit d of *_smem set) or inside its global scratch slice.
struct Layout {
    uint32_t llr_off[kMaxLayers];
    uint32_t llr_words[kMaxLayers];  // capacity in 32-bit words (bounds)
    uint32_t bl_off[kMaxLayers];
    uint32_t br_off[kMaxLayers];
    uint32_t b_words[kMaxLayers];    // capacity of one beta buffer in words
    uint32_t llr_smem, bl_smem, br_smem;
    uint32_t src_off;                // shared: selection scatter area (64 words) and the
                                     //   info-bit buffer (info_words), then 32 frame ids
    uint32_t info_words;             // max(64, ceil(K_info / 32))
    uint32_t ns_off;                 // global: non-systematic transform scratch
    uint32_t ns_words;
    uint32_t smem_per_warp;
    uint32_t gmem_per_warp;
};

// One decode work item: a code, its node schedule and memory layout, a list
// size, and where its frames' inputs and outputs sit.  Every warp copies the
// item of its current task into the head of its shared-memory slice.
struct Item {
    DevCode code;
    const uint32_t *ops;
    int n_ops;
    int root_special;
    Layout lay;
    size_t llr_off;             // batch: offset of the item's first LLR (floats)
    size_t info_off;            // batch: offset of its first info byte
    int status_off;             // batch: index of its first status entry
    int n_frames;               // frames of the item (rows of llr / outputs)
    int L;                      // list size of this stage
    int L_out;                  // pm_out row length
    int stage_L;                // reported in status bits 8..15
    const int32_t *frame_list;  // NULL: frames 0..n_frames-1; else frame ids
    const int32_t *list_count;  // with frame_list: device count of ids
    int32_t *next_list;         // adaptive: failed frames are appended here
    int32_t *next_count;        //   (NULL when this is the last stage)
    const float *llr;
    uint8_t *info_out;
    int32_t *status_out;
    float *pm_out;
    uint32_t *err;              // debug error word (checked builds)
    int llr_cg;                 // 1: read the channel LLRs past L1 (serving loop:
                                //   a persistent kernel may see a reused buffer)
    int quant;                  // number format (serving loop: chosen per context)
};

// bytes reserved at the head of each warp's shared slice for its Item copy,
// followed by the table of its 36 buffer pointers
constexpr uint32_t kItemBytes = (uint32_t)((sizeof(Item) + 15) / 16 * 16);
constexpr uint32_t kPtabBytes = 3 * kMaxLayers * 8;

struct KParams {
    Item single;                // the item when tasks == NULL
    const Item *items;          // batch: device item table
    const int2 *tasks;          // batch: (item, first frame) per task, NULL = single item
    int n_tasks;
    int *task_ctr;              // batch: next task (zeroed before the launch)
    char *gmem;                 // global scratch base
    uint32_t gmem_per_warp;
    uint32_t smem_per_warp;
    int total_warps;
    const float *llr_pool;      // batch pools (items add their offsets)
    uint8_t *info_pool;
    int32_t *status_pool;
    unsigned long long *op_cycles;  // step-profiling builds: 16 x (cycles, steps); else unused
};

// decoder kernel variants (scl_<format>.cu, scl_<format>_nodes.cu): without
// or with the pruned-node handlers, each at a lower occupancy (node-free: 5
// blocks of 4 warps per SM, 96 registers; node-capable: 4 blocks, 128
// registers) or a higher one (7 blocks, 72 registers).  resident_warps is the
// tuned occupancy target: 24 or more selects the higher one.
enum KernelVariant : int { KV_PLAIN = 0, KV_NODES = 1, KV_DENSE = 2, KV_NODES_DENSE = 3 };
inline int kernel_variant(bool nodes, int resident_warps)
{
    const bool hi = resident_warps >= 24;
    return nodes ? (hi ? KV_NODES_DENSE : KV_NODES) : (hi ? KV_DENSE : KV_PLAIN);
}
cudaError_t launch_scl(int quant, int kv, const KParams &p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t scl_func_attrs(int quant, int kv, size_t smem, int block, int *blocks_per_sm);
// the one-path (SC) kernel: warp per frame, single item (sc_kernel.cu)
cudaError_t launch_sc(int quant, const KParams &p, int grid, int block, size_t smem, cudaStream_t s);
cudaError_t sc_attrs(int quant, size_t smem, int block, int *blocks_per_sm);

// ---------------------------------------------------------------------------
// serving loop (server.cu)
struct SrvReq {            // ring entry, written by the host
    int ctx;
    int n;
    const float *llr;
    uint8_t *info;
    int32_t *status;
};
struct SrvComp {           // completion record, written by the device
    unsigned long long t_open, t_end;
    int status;
    uint32_t seq;          // ticket + 1 once complete
};
struct SrvCtl {            // control block in mapped memory
    uint32_t tail;         // tickets published by the host
    uint32_t abort;        // host sets 1 to stop the loop
    int32_t exit_status;   // device: PSCL_ETIMEDOUT when it left on its idle budget
    uint32_t exit_warp;    // device: the warp that found the idle budget spent
    long long exit_idle_ns;            // device: how long it had been idle
    unsigned long long exit_budget_ns; // device: the budget it compared with
    uint32_t exit_opened, exit_head;   // device: tickets opened / oldest open at that time
    uint32_t exit_opening, exit_tail;
};
struct SrvDReq {           // device copy of an open request
    int ctx, n;
    const float *llr;
    uint8_t *info;
    int32_t *status;
    unsigned long long t_open;
};
struct SrvDev {            // device-side counters
    uint32_t opened;       // tickets copied into device memory
    uint32_t opening;      // ticket range being copied (CAS guard)
    uint32_t head;         // oldest ticket that may still have unclaimed frames
    uint32_t abort;        // device copy of the abort word
};

struct SrvParams {
    KParams K;             // items, gmem, gmem_per_warp, smem_per_warp, total_warps
    int n_ctx;
    unsigned quant_mask;   // number formats present among the contexts (bit q)
    SrvCtl *ctl;
    SrvReq *ring;
    SrvComp *comp;
    SrvDev *dev;
    SrvDReq *dreq;
    unsigned long long *claim;   // ticket << 32 | next frame
    uint32_t *done;              // frames finished
    int R;                       // ring slots (power of two)
    unsigned long long idle_ns;
};

// one serving kernel decodes every number format (the item's quant field
// selects the path at run time)
cudaError_t server_attrs(bool nodes, size_t smem, int *blocks_per_sm);
cudaError_t server_launch(bool nodes, const SrvParams &S, int grid, size_t smem, cudaStream_t s);

struct EncParams {
    DevCode code;
    const uint8_t *info;
    uint8_t *x;
    int n_frames;
};
cudaError_t launch_encode(const EncParams &p, cudaStream_t s);

}  // namespace pscl
