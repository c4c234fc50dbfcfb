// server_kernel.cuh -- device-resident serving loop (continuous batching).
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
// Contexts may use different number formats: one kernel holds the float,
// int16 and int8 decoders and each task takes the path of its context.
//
// Every wait is bounded: claims retry a bounded number of times, an idle warp
// sleeps in short steps, and after idle_timeout without any new request the
// first warp to notice records PSCL_ETIMEDOUT and raises the device abort word
// so that every warp leaves together (no warp is left behind that could miss
// a request nobody opens); the host's abort word stops all warps between
// tasks.  Any warp that finds no work opens newly published requests before
// it sleeps, so opening never depends on particular warps being alive.
#pragma once
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

// device nanosecond timer, read as two 32-bit halves with the high half
// checked on both sides of the low one (a read across a carry out of the low
// half returns the later value)
__device__ __forceinline__ unsigned long long gtimer()
{
    uint32_t hi0, lo, hi1;
    asm volatile("mov.u32 %0, %%globaltimer_hi;" : "=r"(hi0));
    asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(lo));
    asm volatile("mov.u32 %0, %%globaltimer_hi;" : "=r"(hi1));
    if (hi1 != hi0) asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(lo));
    return ((unsigned long long)hi1 << 32) | lo;
}

// Idle time of a warp, accumulated from the steps between its own timer
// reads: a step counts at most kIdleStepNs and a timer that reads earlier
// than before counts nothing, so the budget measures time this warp spent
// looking for work, whatever the timer does between two reads.
constexpr long long kIdleStepNs = 20000000;  // 20 ms: far above one loop step
struct IdleClock {
    unsigned long long prev;
    long long idle;
    __device__ void reset() { prev = gtimer(); idle = 0; }
    __device__ long long tick()
    {
        const unsigned long long now = gtimer();
        const long long d = (long long)(now - prev);
        prev = now;
        if (d > 0) idle += d < kIdleStepNs ? d : kIdleStepNs;
        return idle;
    }
};

// copy newly published requests into device memory (one warp at a time).
// `opened` is read before the host's tail and the range is opened only when
// the tail is ahead of it: a warp holding a tail value older than what
// another warp has opened since must not open the range backwards (that
// would walk 2^32 tickets and reset the claims of requests in flight).
static __device__ void srv_open(const SrvParams &S)
{
    const uint32_t op = *(volatile uint32_t *)&S.dev->opened;
    __threadfence();
    const uint32_t t = *(volatile uint32_t *)&S.ctl->tail;
    if ((int)(t - op) <= 0 || (int)(t - op) > S.R) return;
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
static __device__ int srv_try_claim(const SrvParams &S, uint32_t k, unsigned long long w, int n, int fpw)
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

template <bool NODES>
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
#ifdef PSCL_OPPROF
    c.prof = nullptr;
#endif
    int cur = -1;
    IdleClock idle;
    idle.reset();
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
                idle.reset();
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
        if (c.lane == 0 && !stop && k_found < 0) {
            // nothing to claim: open whatever the host has published since
            // (any warp may; the CAS on `opening` lets one copy at a time)
            srv_open(S);
            if (*(volatile uint32_t *)&S.dev->opened != opened) {
                idle.reset();
            } else if (idle.tick() > (long long)S.idle_ns) {
                // idle budget spent: every warp leaves (device abort word)
                if (atomicCAS(&S.ctl->exit_status, 0, PSCL_ETIMEDOUT) == 0) {
                    volatile SrvCtl *ctl = S.ctl;
                    ctl->exit_warp = (uint32_t)gwarp;
                    ctl->exit_idle_ns = idle.idle;
                    ctl->exit_budget_ns = S.idle_ns;
                    ctl->exit_opened = *(volatile uint32_t *)&S.dev->opened;
                    ctl->exit_head = *(volatile uint32_t *)&S.dev->head;
                    ctl->exit_opening = *(volatile uint32_t *)&S.dev->opening;
                    ctl->exit_tail = ctl->tail;
                    __threadfence_system();
                }
                atomicExch(&S.dev->abort, 1u);
                idle_out = 1;
            }
        }
        stop = __shfl_sync(PSCL_FULL, stop, 0);
        idle_out = __shfl_sync(PSCL_FULL, idle_out, 0);
        if (stop || idle_out) break;
        if (k_found < 0) {
            // idle: bounded wait (the budget is checked above); new requests
            // opened just now are scanned without sleeping
            if (__shfl_sync(PSCL_FULL, (int)(*(volatile uint32_t *)&S.dev->opened != opened), 0)) continue;
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
        switch (c.P->quant) {
        case 0: decode_task<QF32, NODES>(c, pos_found, d.n); break;
        case 1: decode_task<QI16, NODES>(c, pos_found, d.n); break;
        default: decode_task<QI8, NODES>(c, pos_found, d.n); break;
        }
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
        if (c.lane == 0) idle.reset();
    }
}

template <bool NODES>
cudaError_t srv_prepare(size_t smem, int *bps)
{
    int dev, optin = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(server_kernel<NODES>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(bps, server_kernel<NODES>, 128, smem);
    return e;
}

template <bool NODES>
cudaError_t srv_launch(const SrvParams &S, int grid, size_t smem, cudaStream_t s)
{
    server_kernel<NODES><<<grid, 128, smem, s>>>(S);
    return cudaGetLastError();
}

}  // namespace pscl
