// server.cu -- device-resident serving loop (continuous batching).
//
// The host appends decode requests to a ring in mapped pinned memory and
// advances a published-ticket counter.  A persistent kernel keeps the code
// contexts (item table), the warps' scratch and the per-request frame
// counters on the GPU.  Its warps open newly published requests (copying
// them into device memory), take tasks of 32/L frames from any open request
// with a ticket-tagged compare-and-swap, decode them exactly like
// pscl_decode, and the warp that finishes a request's last frame writes its
// completion record (device timestamps from %globaltimer) back to mapped
// memory.  Requests that arrive while others are decoding are admitted at
// once and share the warps with them.
//
// Every wait is bounded: claims retry a bounded number of times, an idle warp
// sleeps in short steps and leaves after idle_timeout without work (recording
// PSCL_ETIMEDOUT), and the host's abort word stops all warps between tasks.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>
#include <time.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/polarscl.h"
#include "scl_kernel.cuh"

namespace pscl {

__device__ __forceinline__ unsigned long long gtimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// copy newly published requests into device memory (one warp at a time)
__device__ void srv_open(const SrvParams &S)
{
    const uint32_t t = *(volatile uint32_t *)&S.ctl->tail;
    const uint32_t op = *(volatile uint32_t *)&S.dev->opened;
    if (t == op) return;
    if (atomicCAS(&S.dev->opening, op, t) != op) return;
    __threadfence_system();  // ring entries are read after the published count
    for (uint32_t k = op; k != t; ++k) {
        const int slot = (int)(k & (uint32_t)(S.R - 1));
        volatile SrvReq *r = S.ring + slot;
        SrvDReq d;
        d.ctx = r->ctx;
        d.n = r->n;
        d.llr = (const float *)r->llr;
        d.info = (uint8_t *)r->info;
        d.status = (int32_t *)r->status;
        d.t_open = gtimer();
        S.dreq[slot] = d;
        S.done[slot] = 0;
        S.claim[slot] = (unsigned long long)k << 32;
    }
    __threadfence();
    atomicExch(&S.dev->opened, t);
}

// try to claim fpw frames of ticket k whose claim word was just read as w
// (tag k, next frame below n): a few compare-and-swaps, each retry using the
// value the failed swap returned; -1 when others took everything first or
// kept winning (the caller moves on to other requests)
__device__ int srv_try_claim(const SrvParams &S, uint32_t k, unsigned long long w, int n, int fpw)
{
    const int slot = (int)(k & (uint32_t)(S.R - 1));
    for (int tries = 0; tries < 4; ++tries) {
        if ((uint32_t)(w >> 32) != k) return -1;
        const int pos = (int)(uint32_t)w;
        if (pos >= n) return -1;
        const unsigned long long old = atomicCAS(&S.claim[slot], w, w + (unsigned long long)fpw);
        if (old == w) return pos;
        w = old;
    }
    return -1;
}

template <class Qt, bool NODES>
__global__ void __launch_bounds__(128, 4) server_kernel(const __grid_constant__ SrvParams S)
{
    extern __shared__ __align__(16) char smem[];
    const KParams &K = S.K;
    Ctx c;
    const int warp = threadIdx.x >> 5;
    c.lane = threadIdx.x & 31;
    const int gwarp = blockIdx.x * (blockDim.x >> 5) + warp;
    c.sm = smem + (size_t)warp * K.smem_per_warp;
    c.gm = K.gmem + (size_t)gwarp * K.gmem_per_warp;
    c.P = (const Item *)c.sm;
    int cur = -1;
    unsigned long long last_work = gtimer();
    uint32_t seen_opened = 0;
    unsigned sleep_ns = 128;
    const bool poller = (gwarp & 7) == 0;   // a few warps watch the host words
    for (;;) {
        // --- find a task: the 32 lanes look at 32 open requests at a time
        int k_found = -1, pos_found = -1, stop = 0, idle_out = 0;
        uint32_t opened = 0, head = 0;
        if (c.lane == 0) {
            if (poller) {
                if (*(volatile uint32_t *)&S.ctl->abort) atomicExch(&S.dev->abort, 1u);
                srv_open(S);
            }
            stop = *(volatile uint32_t *)&S.dev->abort ? 1 : 0;
            opened = *(volatile uint32_t *)&S.dev->opened;
            head = *(volatile uint32_t *)&S.dev->head;
            if (opened != seen_opened) {
                // new requests anywhere keep every warp alive
                seen_opened = opened;
                last_work = gtimer();
            }
        }
        stop = __shfl_sync(PSCL_FULL, stop, 0);
        if (stop) break;
        opened = __shfl_sync(PSCL_FULL, opened, 0);
        head = __shfl_sync(PSCL_FULL, head, 0);
        __threadfence();
        for (uint32_t base = head; base != opened && (int)(base - head) < S.R; base += 32) {
            if (c.lane == 0) stop = *(volatile uint32_t *)&S.dev->abort ? 1 : 0;
            stop = __shfl_sync(PSCL_FULL, stop, 0);
            if (stop) break;
            const uint32_t k = base + (uint32_t)c.lane;
            const bool valid = (int)(k - base) < (int)(opened - base) && (int)(k - head) < S.R;
            bool claimable = false, finished = false;  // lanes past `opened` never count
            unsigned long long w = 0;
            int n = 0, fpw = 1;
            if (valid) {
                const int slot = (int)(k & (uint32_t)(S.R - 1));
                w = *(volatile unsigned long long *)&S.claim[slot];
                const volatile SrvDReq *d = S.dreq + slot;
                const int ctx = d->ctx;
                n = d->n;
                if ((uint32_t)(w >> 32) != k || (int)(uint32_t)w >= n) {
                    finished = true;  // every frame taken (or the slot moved on)
                } else if (ctx >= 0 && ctx < S.n_ctx) {
                    claimable = true;
                    fpw = 32 / S.K.items[ctx].L;
                }
            }
            // requests from the head whose frames are all taken: move the head
            const uint32_t fin = __ballot_sync(PSCL_FULL, finished);
            const int run = fin == 0xFFFFFFFFu ? 32 : __ffs(~fin) - 1;
            if (c.lane == 0 && base == head && run > 0) {
                atomicMax(&S.dev->head, base + (uint32_t)run);
            }
            uint32_t cand = __ballot_sync(PSCL_FULL, claimable);
            while (cand) {
                const int l = __ffs(cand) - 1;
                int pos = -1;
                if (c.lane == l) pos = srv_try_claim(S, k, w, n, fpw);
                pos = __shfl_sync(PSCL_FULL, pos, l);
                if (pos >= 0) {
                    k_found = (int)__shfl_sync(PSCL_FULL, k, l);
                    pos_found = pos;
                    break;
                }
                cand &= cand - 1u;
            }
            if (k_found >= 0) break;
        }
        if (c.lane == 0 && !stop && k_found < 0 && gtimer() - last_work > S.idle_ns) {
            atomicCAS(&S.ctl->exit_status, 0, PSCL_ETIMEDOUT);
            idle_out = 1;
        }
        stop = __shfl_sync(PSCL_FULL, stop, 0);
        idle_out = __shfl_sync(PSCL_FULL, idle_out, 0);
        if (stop || idle_out) break;
        if (k_found < 0) {
            // idle: bounded wait (the budget is checked above)
            __nanosleep(sleep_ns);
            sleep_ns = sleep_ns < 4096 ? sleep_ns * 2 : 4096;
            continue;
        }
        sleep_ns = 128;
        const int slot = k_found & (S.R - 1);
        // the slot is rewritten by whichever warp opens the ticket that reuses
        // it: read it past this SM's L1, which may still hold the request the
        // slot carried before
        SrvDReq d;
        {
            const volatile SrvDReq *vd = S.dreq + slot;
            d.ctx = vd->ctx;
            d.n = vd->n;
            d.llr = vd->llr;
            d.info = vd->info;
            d.status = vd->status;
            d.t_open = vd->t_open;
        }
        if (d.ctx != cur) {
            load_item(c, K.items + d.ctx, K, false);
            cur = d.ctx;
        }
        if (c.lane == 0) {
            Item *it = (Item *)c.sm;
            it->llr = d.llr;
            it->info_out = d.info;
            it->status_out = d.status;
            it->pm_out = nullptr;
            it->n_frames = d.n;
        }
        __syncwarp();
        decode_task<Qt, NODES>(c, pos_found, d.n);
        if (c.lane == 0) {
            const int cnt = d.n - pos_found < c.fpw ? d.n - pos_found : c.fpw;
            __threadfence();
            const uint32_t prev = atomicAdd(&S.done[slot], (uint32_t)cnt);
            if ((int)prev + cnt == d.n) {
                // last frame of the request: publish its completion
                __threadfence_system();
                volatile SrvComp *cp = S.comp + slot;
                cp->t_open = d.t_open;
                cp->t_end = gtimer();
                cp->status = 0;
                __threadfence_system();
                cp->seq = (uint32_t)k_found + 1u;
                __threadfence_system();
            }
        }
        __syncwarp();
        if (c.lane == 0) last_work = gtimer();
    }
}

static std::mutex g_srv_attr_mu;

template <class Qt, bool NODES>
static cudaError_t srv_prepare(size_t smem, int *bps)
{
    std::lock_guard<std::mutex> lk(g_srv_attr_mu);
    int dev, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(server_kernel<Qt, NODES>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, server_kernel<Qt, NODES>, 128, smem);
    return e;
}

template <class Qt, bool NODES>
static cudaError_t srv_launch(const SrvParams &S, int grid, size_t smem, cudaStream_t s)
{
    server_kernel<Qt, NODES><<<grid, 128, smem, s>>>(S);
    return cudaGetLastError();
}

cudaError_t server_attrs(int quant, bool nodes, size_t smem, int *bps)
{
    if (quant == 0) return nodes ? srv_prepare<QF32, true>(smem, bps) : srv_prepare<QF32, false>(smem, bps);
    if (quant == 1) return nodes ? srv_prepare<QI16, true>(smem, bps) : srv_prepare<QI16, false>(smem, bps);
    return nodes ? srv_prepare<QI8, true>(smem, bps) : srv_prepare<QI8, false>(smem, bps);
}

cudaError_t server_launch(int quant, bool nodes, const SrvParams &S, int grid, size_t smem, cudaStream_t s)
{
    if (quant == 0) return nodes ? srv_launch<QF32, true>(S, grid, smem, s) : srv_launch<QF32, false>(S, grid, smem, s);
    if (quant == 1) return nodes ? srv_launch<QI16, true>(S, grid, smem, s) : srv_launch<QI16, false>(S, grid, smem, s);
    return nodes ? srv_launch<QI8, true>(S, grid, smem, s) : srv_launch<QI8, false>(S, grid, smem, s);
}

}  // namespace pscl
