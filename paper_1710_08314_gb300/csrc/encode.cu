// encode.cu -- polar encoder (Sec. II-A): u_A = (data || CRC), x = u F, and for
// systematic codes x = (u F with the frozen part zeroed) F.  One warp per
// frame; the frame's N bits live in shared memory as 32-bit words.
#include <cuda_runtime.h>
#include <stdint.h>

#include "internal.h"

namespace pscl {

constexpr int kEncWarps = 4;

__device__ void transform_words(uint32_t *u, int N, int lane)
{
    const int NW = N >= 32 ? N >> 5 : 1;
    // position strides >= 32: x_i ^= x_{i+s} on whole words
    for (int sw = NW >> 1; sw >= 1; sw >>= 1) {
        for (int w = lane; w < NW; w += 32)
            if ((w & sw) == 0) u[w] ^= u[w + sw];
        __syncwarp();
    }
    // strides < 32 inside a word
    const int top = N < 32 ? N : 32;
    const uint32_t lo[5] = {0x55555555u, 0x33333333u, 0x0F0F0F0Fu, 0x00FF00FFu, 0x0000FFFFu};
    for (int w = lane; w < NW; w += 32) {
        uint32_t v = u[w];
#pragma unroll
        for (int k = 0; k < 5; ++k)
            if ((1 << k) < top) v ^= (v >> (1 << k)) & lo[k];
        u[w] = v;
    }
    __syncwarp();
}

__global__ void __launch_bounds__(32 * kEncWarps) encode_kernel(const EncParams P)
{
    extern __shared__ uint32_t esm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int frame = blockIdx.x * kEncWarps + warp;
    if (frame >= P.n_frames) return;
    const DevCode &cd = P.code;
    const int N = cd.N, NW = N >= 32 ? N >> 5 : 1;
    uint32_t *u = esm + warp * NW;  // the frame's N bits (NW words per warp)
    const int nbytes = (cd.kinfo + 7) >> 3;
    const uint8_t *info = P.info + (size_t)frame * (size_t)nbytes;
    // CRC of the data bits, MSB first (one lane; bytes through the table)
    uint32_t crc = 0;
    if (lane == 0 && cd.crc_len > 0) {
        uint32_t reg = 0;
        const int full = cd.kinfo >> 3;
        for (int b = 0; b < full; ++b) reg = (reg << 8) ^ __ldg(&cd.crc_lut[(reg >> 24) ^ info[b]]);
        for (int k = full * 8; k < cd.kinfo; ++k) {
            const uint32_t bit = (info[k >> 3] >> (7 - (k & 7))) & 1u;
            const uint32_t top = reg >> 31;
            reg <<= 1;
            if (top ^ bit) reg ^= cd.poly32;
        }
        crc = reg >> (32 - cd.crc_len);
    }
    crc = __shfl_sync(0xFFFFFFFFu, crc, 0);
    // u: information positions take data bits then CRC bits in order
    for (int w = lane; w < NW; w += 32) {
        int k = 0;
        for (int v = 0; v < w; ++v) k += __popc(__ldg(&cd.amask[v]));
        uint32_t am = __ldg(&cd.amask[w]), word = 0;
        while (am) {
            const int b = __ffs(am) - 1;
            am &= am - 1u;
            uint32_t bit;
            if (k < cd.kinfo) bit = (info[k >> 3] >> (7 - (k & 7))) & 1u;
            else bit = (crc >> (cd.crc_len - 1 - (k - cd.kinfo))) & 1u;
            word |= bit << b;
            ++k;
        }
        u[w] = word;
    }
    __syncwarp();
    transform_words(u, N, lane);
    if (cd.systematic) {
        for (int w = lane; w < NW; w += 32) u[w] &= __ldg(&cd.amask[w]);
        __syncwarp();
        transform_words(u, N, lane);
    }
    uint8_t *x = P.x + (size_t)frame * (size_t)N;
    for (int i = lane; i < N; i += 32) x[i] = (uint8_t)((u[i >> 5] >> (i & 31)) & 1u);
}

cudaError_t launch_encode(const EncParams &p, cudaStream_t s)
{
    const int grid = (p.n_frames + kEncWarps - 1) / kEncWarps;
    const int NW = p.code.N >= 32 ? p.code.N >> 5 : 1;
    encode_kernel<<<grid, 32 * kEncWarps, (size_t)kEncWarps * NW * sizeof(uint32_t), s>>>(p);
    return cudaGetLastError();
}

}  // namespace pscl
