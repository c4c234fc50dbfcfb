/*
 * polarscl.h -- C ABI of the GB300 polar list decoder (libpolarscl.so).
 *
 * Batched successive-cancellation list decoding of polar codes with CRC aid,
 * tree pruning, fixed-point LLRs and adaptive list schedules, after Leonardon
 * et al., "Fast and Flexible Software Polar List Decoders" (SCL in Sec. II-B
 * and Algorithm 1; genericity and flexibility in Sec. III; CRC, sorting and
 * partial sums in Sec. IV).
 *
 * Conventions shared by every call:
 *  - A code has length N = 2^n (8 <= N <= 8192), |A| = K information
 *    positions that INCLUDE the c CRC bits (K_info = K - c data bits).  Data
 *    bits then CRC bits fill A in increasing position order.  The CRC is the
 *    MSB-first remainder of the data bits times x^c modulo x^c + crc_poly
 *    (initial value 0, no reflection, no final XOR).
 *  - Encoding (Sec. II-A): x = u F^{(x)n}, F = [[1,0],[1,1]]; systematic codes
 *    re-encode after zeroing the frozen part so that x_A = u_A.
 *  - LLRs are ln P(x=0)/P(x=1); BPSK maps 0 -> +1.  A frame's LLR row holds
 *    the N - P transmitted positions in increasing position order; punctured
 *    positions get LLR 0 inside the decoder.
 *  - Bit vectors passed as bytes are packed MSB first: bit i is bit 7 - (i&7)
 *    of byte i >> 3.
 *  - Every device buffer belongs to the caller.  Calls are asynchronous on the
 *    given CUDA stream (a cudaStream_t passed as void*, NULL = legacy default
 *    stream) and return after enqueueing.  Argument errors are reported
 *    before anything is enqueued.
 *  - Return value: PSCL_OK (0) or a negative PSCL_E* code; pscl_last_error()
 *    returns a message for the calling thread's last failure.
 */
#ifndef POLARSCL_H
#define POLARSCL_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PSCL_OK 0
#define PSCL_EINVAL (-1)       /* an argument is out of range */
#define PSCL_ENOMEM (-2)       /* a device or host allocation failed */
#define PSCL_EUNSUPPORTED (-3) /* valid, but not supported by the kernels */
#define PSCL_ECUDA (-4)        /* a CUDA call failed (message has the details) */
#define PSCL_ETIMEDOUT (-5)    /* a bounded wait ran out */
#define PSCL_EAGAIN (-6)       /* a queue is full; retry later */

typedef struct pscl_code_s *pscl_code;

/* Decoding algorithms (Sec. II-B): SC is the list of one; CASCL keeps L paths
 * and picks the best-metric candidate that passes the CRC (Sec. IV-B);
 * FASCL decodes with L = 1, 2, 4, ..., L and stops at the first CRC pass;
 * PASCL decodes with L = 1 and then directly with L.                        */
typedef enum { PSCL_SC = 0, PSCL_CASCL = 1, PSCL_PASCL = 2, PSCL_FASCL = 3 } pscl_algo;

/* LLR and metric representation (Sec. III-B-3).  Input LLRs are always float;
 * the fixed-point paths quantise q = clamp(rint_half_even(llr * 2^f), -Q, Q)
 * with (f, Q) = (5, 32767) for I16 and (2, 127) for I8, and saturate every
 * addition to [-Q, Q]; their metrics are normalised by subtracting the
 * smallest active metric after every step.                                 */
typedef enum { PSCL_F32 = 0, PSCL_I16 = 1, PSCL_I8 = 2 } pscl_quant;

#define PSCL_PRUNE_R0 1u
#define PSCL_PRUNE_R1 2u
#define PSCL_PRUNE_REP 4u
#define PSCL_PRUNE_SPC 8u

/* Tree pruning (Sec. II-B, Sec. III-B-2): the top-most node whose leaves are
 * all frozen (R0), all information (R1), all frozen but the last (REP) or
 * only the first frozen (SPC) is decoded as a whole if its type is enabled
 * in `mask` and its size is within the limit; precedence R0 > R1 > REP > SPC.
 * rep_max: 0 = no limit (REP2+), 8 = REP8-.  spc_max: 4 = SPC4 (size 4
 * only), 0 = no limit (SPC4+).  r1_max: 0 = no limit.  r1_t / spc_t: how many
 * least-reliable positions the R1 / SPC candidates flip (r1_t = 2 is the
 * paper's Chase-2, Sec. IV-C); the kernels accept 1 <= r1_t <= 3 and
 * 1 <= spc_t <= 4.  node_min: the smallest node of two or more leaves that
 * is pruned (0, 1 or 2 = any size, the paper's setting); smaller nodes are
 * decoded leaf by leaf, where the GPU decodes them inside its register
 * subtrees (node_min = 2 x fusion size + 1 keeps every register subtree
 * whole).  mask = 0 decodes the full tree leaf by leaf.                    */
typedef struct {
    uint32_t mask;
    int rep_max;
    int spc_max;
    int r1_t;
    int spc_t;
    int r1_max;
    int node_min;
} pscl_pruning;

/* Create a code descriptor and upload it to the current CUDA device.
 * frozen: host, N bytes, nonzero = frozen; exactly N - K of them.
 * crc_len: 0..32 (any length: standard and custom CRCs, Sec. III-A);
 * crc_poly: generator without its top bit, below 2^crc_len (e.g. 0x07,
 * 0x1021, 0x04C11DB7, or 0x864CFB for a 24-bit CRC); crc_len <= K.
 * N up to 8192: the decoder's slot tables cover schedule depths up to 12,
 * which N = 8192 reaches only with register subtrees of 2 or more leaves
 * (the default); a deeper schedule is refused with PSCL_EUNSUPPORTED.
 * puncture: host, N bytes, nonzero = not transmitted, or NULL.
 * systematic: 1 for systematic encoding (the paper's), 0 for x = u F.
 * On success *out owns device memory until pscl_destroy_code.
 * Errors: PSCL_EINVAL (bad N, K, counts, CRC), PSCL_ENOMEM, PSCL_ECUDA.   */
int pscl_create_code(int N, int K, const uint8_t *frozen, int crc_len, uint32_t crc_poly,
                     const uint8_t *puncture, int systematic, pscl_code *out);

/* Free a descriptor.  The caller must make sure no queued work still uses
 * it (e.g. synchronise the streams it was used on).                        */
int pscl_destroy_code(pscl_code code);

/* Query code parameters (any pointer may be NULL).                          */
int pscl_code_info(pscl_code code, int *N, int *K, int *K_info, int *n_punctured);

/* Build (once per pruning setting) the node schedules the kernels walk for
 * this code -- for the default and every tuned register-subtree size, in
 * their float and fixed-point forms -- and cache them with the code.
 * pscl_decode builds what it needs itself; call this first when decodes will
 * be captured in a CUDA graph or use pscl_decode_static, because a build
 * makes a synchronous upload.                                               */
int pscl_prepare(pscl_code code, const pscl_pruning *pruning);

/* Record measured tuning for decodes of this code with list size L, number
 * format quant and pruning (NULL or mask 0 = the unpruned entry, anything
 * else = the pruned entry): warps_per_sm (1..64) sizes each warp's shared-memory
 * slice as if that many warps shared an SM (more warps hide more latency,
 * fewer keep more LLR layers on chip; sizing for more warps than are
 * resident leaves the rest of the SM's shared memory to the L1 cache);
 * fuse_leaves (1, 2, 4, 8) is the largest unpruned subtree decoded in
 * registers; warps_per_block (1, 2, 4, 8; 0 = 4) sets the frames a block
 * holds (warps x 32/L) and so the granularity of shared-memory allocation
 * and of block scheduling; resident_warps (0..64; 0 = warps_per_sm) picks
 * the decoder's register cap: 24 or more selects the 72-register variant
 * (up to 28 warps per SM), less the 96-register (node-free, 20 warps) or
 * 128-register (node-capable, 16 warps) one.  (0, 0, 0, 0) restores the
 * defaults (32 warps, the pscl_set_fusion size, 4 warps per block).  Results never depend
 * on the tuning.  Written by the package's autotuner.                      */
int pscl_code_tune(pscl_code code, int L, pscl_quant quant, const pscl_pruning *pruning, int warps_per_sm,
                   int fuse_leaves, int warps_per_block, int resident_warps);

/* Decode n_frames frames (Algorithm 1 with the selected algorithm).
 * llr: device, n_frames x (N - P) float32, row-major.
 * L: list size (maximum list size for FASCL/PASCL), one of 1, 2, 4, 8, 16, 32.
 * pruning: NULL = no pruning.
 * info_out: device, n_frames x ceil(K_info / 8) bytes, packed MSB first.
 * status_out: device, int32 per frame: bit 0 = the output passed the CRC
 *   (always 1 when crc_len = 0), bits 8..15 = list size of the stage that
 *   produced it, bits 16..23 = its path slot.
 * pm_out: device or NULL; n_frames x L float32 path metrics of the final
 *   stage in slot order (fixed point converted exactly), +inf for unused
 *   slots.
 * The library keeps a scratch workspace per (device, stream) that it grows
 * on demand (a cudaMalloc, after waiting for the stream's queued work when it
 * replaces a smaller one): call once outside stream capture before capturing,
 * or use pscl_decode_ws.  Calls on one stream share its workspace in stream
 * order; calls on different streams use different workspaces and may run
 * concurrently.                                                              */
int pscl_decode(pscl_code code, const float *llr, int n_frames, int L, pscl_algo algo,
                const pscl_pruning *pruning, pscl_quant quant, uint8_t *info_out,
                int32_t *status_out, float *pm_out, void *stream);

/* pscl_decode from host buffers, with the transfers overlapped (no
 * counterpart in the paper: its decoder reads host memory directly).
 * llr_host: host, n_frames x (N - P) float32, row-major; info_host: host,
 * n_frames x ceil(K_info / 8) bytes; status_host: host, int32 per frame
 * (layouts as pscl_decode).  Page-locked host buffers let the copies run
 * asynchronously; pageable ones work but each copy then waits for itself.
 * Batches of 8192 frames or more are cut into up to four chunks: one
 * internal stream copies the chunks in while two others decode them
 * alternately and copy each chunk's outputs back, so transfers and decodes
 * of different chunks overlap.  Everything is ordered after the work
 * already queued on `stream`, and later work on `stream` waits for all of
 * it: synchronize `stream` before reading the outputs.  The library keeps,
 * per (device, stream), the internal streams, events and a device staging
 * buffer (grown on demand; growing waits for that stream's earlier calls).
 * Not for stream capture.  Errors: as pscl_decode, all argument errors
 * before anything is enqueued.                                              */
int pscl_decode_host(pscl_code code, const float *llr_host, int n_frames, int L, pscl_algo algo,
                     const pscl_pruning *pruning, pscl_quant quant, uint8_t *info_host,
                     int32_t *status_host, void *stream);

/* Bytes of device workspace pscl_decode_ws needs for this call shape.       */
int pscl_workspace_size(pscl_code code, int n_frames, int L, pscl_algo algo,
                        const pscl_pruning *pruning, pscl_quant quant, size_t *bytes);

/* pscl_decode with a caller-provided workspace (device, 256-byte aligned, at
 * least pscl_workspace_size bytes); allocates nothing.                      */
int pscl_decode_ws(pscl_code code, const float *llr, int n_frames, int L, pscl_algo algo,
                   const pscl_pruning *pruning, pscl_quant quant, uint8_t *info_out,
                   int32_t *status_out, float *pm_out, void *workspace, size_t workspace_bytes,
                   void *stream);

/* pscl_decode without any allocation, for callers that cannot allocate device
 * memory while they decode (a real-time receive loop that must never
 * synchronise the device, a process whose device memory belongs to another
 * allocator, work that is set up once and afterwards only launched).  The
 * paper has no counterpart; this is a deployment variant of pscl_decode.
 * Same arguments and results as pscl_decode.  Scratch: a static device array
 * of 32 MiB inside the library, held by every GPU that loads the library
 * until the process exits and shared by all calls, so calls that overlap on
 * the GPU race (serialise them on one stream).  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress); make that first
 * call before any stream capture.  The node schedule must already exist:
 * call pscl_prepare(code, pruning) at set-up (it allocates there).
 * The schedule is looked up for the code's current tuning: after
 * pscl_code_tune, pscl_set_fusion or pscl_set_tuning changes it, call
 * pscl_prepare again (the autotuner does so for the codes it tunes).
 * Errors: PSCL_EINVAL when the schedule is not prepared or when one block's
 * per-warp scratch plus the adaptive frame lists (8 bytes per frame) exceed
 * 32 MiB; otherwise as pscl_decode.                                         */
int pscl_decode_static(pscl_code code, const float *llr, int n_frames, int L, pscl_algo algo,
                       const pscl_pruning *pruning, pscl_quant quant, uint8_t *info_out,
                       int32_t *status_out, float *pm_out, void *stream);

/* Encode n_frames frames (Sec. II-A): info: device, n_frames x
 * ceil(K_info/8) bytes packed MSB first; x_out: device, n_frames x N bytes,
 * one codeword bit (0/1) per byte, punctured positions included.           */
int pscl_encode(pscl_code code, const uint8_t *info, int n_frames, uint8_t *x_out, void *stream);

/* ---------------------------------------------------------------------------
 * Uneven batches (many codes, list sizes and number formats at once).
 * A work item names a code, its frame count, list size, algorithm (PSCL_SC
 * or PSCL_CASCL), number format and pruning (NULL = none, copied at
 * pscl_batch_create), and where its frames sit in three caller pools:
 * llr_offset (floats) of its first LLR row in the LLR pool (rows of N - P
 * floats), info_offset (bytes) of its first output row in the info pool (rows
 * of ceil(K_info/8) bytes), status_offset of its first status entry.       */
typedef struct {
    pscl_code code;
    int n_frames;
    int L;
    pscl_algo algo;
    pscl_quant quant;
    const pscl_pruning *pruning;
    size_t llr_offset;
    size_t info_offset;
    size_t status_offset;
} pscl_work_item;

typedef struct pscl_batch_s *pscl_batch;

/* Plan a batch: uploads an item table and a task list (a task = 32/L frames
 * of one item, longest tasks first) and allocates the scratch of every
 * resident warp.  The codes must outlive the plan.  Allocates (set-up).    */
int pscl_batch_create(const pscl_work_item *items, int n_items, pscl_batch *out);
int pscl_batch_destroy(pscl_batch batch);

/* Decode the whole batch: one persistent launch per number format present;
 * each warp takes the next task from a device counter.  Allocates nothing,
 * so it can be captured in a CUDA graph and replayed with new pool contents.
 * Calls of one plan must not overlap (they share its scratch).             */
int pscl_batch_run(pscl_batch batch, const float *llr_pool, uint8_t *info_pool, int32_t *status_pool,
                   void *stream);

/* The same decode as one launch per work item (the plain form the persistent
 * launch is compared with); identical results.                             */
int pscl_batch_run_plain(pscl_batch batch, const float *llr_pool, uint8_t *info_pool,
                         int32_t *status_pool, void *stream);

/* Launches per run, total tasks and scratch bytes of a plan.                */
int pscl_batch_info(pscl_batch batch, int *n_launches, int *n_tasks, size_t *scratch_bytes);

/* ---------------------------------------------------------------------------
 * Serving loop: a device-resident request loop with continuous batching.
 * The server keeps its decoding contexts (code, list size, pruning and
 * number format per context) and all frame state on the GPU and runs one
 * persistent kernel on its own stream.  Requests are published through a
 * ring in mapped host memory; the kernel's warps take 32/L-frame tasks from
 * every open request, so requests that arrive while others decode share the
 * GPU with them at once.  Results equal pscl_decode's (CASCL, or SC for
 * L = 1) frame by frame.  Admission (pscl_server_submit) needs a free ring
 * slot, room in the frame budget and, with a byte budget, room in it for the
 * request's device footprint (pscl_server_context_info); otherwise the
 * request is deferred with PSCL_EAGAIN.  Every device-side wait is bounded:
 * after idle_timeout_ms without any new request the kernel exits by itself,
 * pscl_server_status reports PSCL_ETIMEDOUT and requests it never finished
 * come back from pscl_server_poll with status PSCL_ETIMEDOUT;
 * pscl_server_stop raises an abort word that the warps check between tasks.
 * While a server runs, wait on streams or events only: a device-wide
 * synchronisation (cudaDeviceSynchronize, and cudaFree, which implies one)
 * waits for the serving kernel itself, which ends only on stop or its idle
 * budget.  For the same reason the library defers its own frees on a device
 * (pscl_destroy_code, pscl_batch_destroy, a replaced decode workspace) while
 * a server runs there, and carries them out when the last one stops.      */
typedef struct pscl_server_s *pscl_server;

typedef struct {
    pscl_code code;
    int L;
    const pscl_pruning *pruning;  /* NULL = none (read at start only) */
    pscl_quant quant;             /* number format of this context */
} pscl_context;

typedef struct {
    const pscl_context *contexts;
    int n_contexts;
    int ring_slots;               /* requests in flight at most, power of two */
    int max_frames_per_request;
    long long max_inflight_frames;/* admission budget (frames); 0 = ring x max */
    long long hbm_budget_bytes;   /* admission budget (device bytes of the
                                     frames in flight); 0 = none */
    int idle_timeout_ms;          /* device loop exits after this long idle */
    int max_warps;                /* 0 = every resident warp */
} pscl_server_cfg;

/* A request: context index, frame count and DEVICE buffers whose contents
 * are ready when pscl_server_submit is called (llr: n_frames x (N - P)
 * floats; info_out: n_frames x ceil(K_info/8) bytes; status_out: int32 per
 * frame, as in pscl_decode).                                               */
typedef struct {
    int context;
    int n_frames;
    const float *llr;
    uint8_t *info_out;
    int32_t *status_out;
} pscl_request;

typedef struct {
    uint64_t ticket;
    int status;                   /* 0 = decoded */
    int n_frames;
    uint64_t t_submit_ns;         /* host CLOCK_MONOTONIC at submit */
    uint64_t t_done_ns;           /* host CLOCK_MONOTONIC when polled complete */
    uint64_t device_ns;           /* device time from opening to last frame */
} pscl_completion;

/* Allocates the server's device and mapped memory and launches its kernel. */
int pscl_server_start(const pscl_server_cfg *cfg, pscl_server *out);
/* Thread-safe, non-blocking.  PSCL_EAGAIN when the ring, the frame budget or
 * the byte budget is full (nothing is dropped; retry), PSCL_EINVAL for a
 * malformed request or one larger than the whole byte budget.              */
int pscl_server_submit(pscl_server s, const pscl_request *req, uint64_t *ticket);
/* Collect up to max completed requests (non-blocking).                     */
int pscl_server_poll(pscl_server s, pscl_completion *out, int max, int *n_out);
/* Footprint of a context: the shared-memory slice and the global scratch
 * slice its decode layout needs per warp (the server's warps hold the largest
 * of each), and the device bytes one of its frames holds while in flight --
 * its LLR row, its output row and status word, and its share (L/32) of a
 * warp's scratch slice.  A request of n frames is charged n times that
 * against hbm_budget_bytes until it completes.  Any pointer may be NULL.    */
int pscl_server_context_info(pscl_server s, int context, size_t *smem_per_warp, size_t *scratch_per_warp,
                             size_t *bytes_per_frame);
/* running: kernel still resident; device_status: PSCL_ETIMEDOUT once it left
 * on its idle budget.                                                       */
int pscl_server_status(pscl_server s, int *running, int *device_status, uint64_t *completed,
                       long long *frames_in_flight);
/* Raise the abort word and wait (at most timeout_ms) for the kernel to end,
 * then free everything; PSCL_ETIMEDOUT keeps the resources.                 */
int pscl_server_stop(pscl_server s, int timeout_ms);

/* Process-wide defaults, used where a code has no pscl_code_tune entry and
 * by every batch and server (no counterpart in the paper: GPU scheduling).
 * pscl_set_tuning: resident warps per SM the shared-memory slices are sized
 *   for, 1..64 (default 32: 28 warps reside, the rest of the shared memory
 *   serves as L1 cache); 24 and more select the 72-register decoder
 *   variants.
 * pscl_set_fusion: largest register subtree, 1, 2, 4 or 8 leaves (1 =
 *   none; 0, the default, = by number format: 4 leaves in float, 2 in fixed
 *   point).  Not thread-safe against concurrent decodes; results never
 *   depend on either.  PSCL_EINVAL outside the ranges.                      */
int pscl_set_tuning(int target_warps_per_sm);
int pscl_set_fusion(int max_leaves);
/* pscl_set_sc_kernel: 1 (default) decodes one-path stages (PSCL_SC, and the
 * first stage of PSCL_FASCL and PSCL_PASCL) of batches up to six waves of
 * resident warps in float (two and a half in fixed point; about 22 k and
 * 12 k frames at N = 2048) with a warp per frame and all of a frame's LLR layers and
 * partial sums in shared memory (lowest latency); larger batches, and every
 * batch with 0, go to the list kernel, which decodes 32 such frames per warp
 * (highest throughput).  Results are identical; not thread-safe against
 * concurrent decodes.                                                       */
int pscl_set_sc_kernel(int enable);

/* Test hooks.  pscl_debug_last_launches: kernel launches of the calling
 * process's most recent decode or batch run.  pscl_debug_error_word: the
 * bounds-check word of the current device's library workspace (non-zero only
 * in the checked build, after an out-of-range access was caught and
 * skipped); *out = 0 when no workspace exists.  pscl_debug_checked: 1 in
 * the checked build, else 0.                                                */
int pscl_debug_last_launches(void);
/* pscl_debug_server_exit: for a serving loop that left on its idle budget,
 * the warp that found the budget spent, how long it had been idle and the
 * budget it compared with (ns), and tickets[4] = (opened, oldest open,
 * being opened, published) at that moment.  Any pointer may be NULL.       */
int pscl_debug_server_exit(pscl_server s, int *warp, long long *idle_ns, unsigned long long *budget_ns,
                           uint32_t *tickets);
/* pscl_debug_server_slots: after the serving kernel has ended, its per-slot
 * device state (claim word, frames done, frame count; ring_slots entries
 * each) and the ticket the host holds outstanding in each slot (~0 = free). */
int pscl_debug_server_slots(pscl_server s, uint64_t *claim, uint32_t *done, int32_t *nframes, uint64_t *tickets);
int pscl_debug_error_word(uint32_t *out);
int pscl_debug_checked(void);
/* pscl_debug_step_cycles: in the step-profiling build (PSCL_OPPROF=1, built
 * as libpolarscl_opprof.so), the list kernel's lane 0 of every warp adds the
 * SM cycles of each schedule step to a per-device counter by category: out
 * receives 16 (cycles, steps) pairs, categories 0..6 the opcodes F, G, leaf
 * or node, h, register subtree, register-subtree pair, 16-leaf quad; 7 + the
 * node type (8 R0, 9 R1, 10 REP, 11 SPC) for pruned nodes; 12 loading a
 * task's frames; 13 the final CRC selection and output; 14 the two-candidate
 * selections that took the general (sorting) path, already inside the
 * categories of their steps.  reset != 0 zeroes
 * the counters after reading.  Other builds return PSCL_EUNSUPPORTED.       */
int pscl_debug_step_cycles(uint64_t *out, int reset);

/* Message for the calling thread's most recent error ("" if none).         */
const char *pscl_last_error(void);

/* Library version string.                                                   */
const char *pscl_version(void);

#ifdef __cplusplus
}
#endif
#endif
