// common.cuh -- shared device helpers of librosen: the Philox4x32-10 stream,
// uniform conversion, status handling.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "rosen.h"

namespace rosen {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two
// 32x32->64 multiplies with xor-mixing of the high halves into the other
// words, the 64-bit key advanced by the two Weyl constants between rounds.
// Counter = (chain, ensemble, step, slot); key = (seed_lo, seed_hi).  It
// replaces the paper's per-thread cuRAND state (Section 3.2): a chain's draws
// are a pure function of its indices, so no state is stored or initialised.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox(uint4 c, uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = c.x * 0xD2511F53u;
        const uint32_t hi0 = __umulhi(c.x, 0xD2511F53u);
        const uint32_t lo1 = c.z * 0xCD9E8D57u;
        const uint32_t hi1 = __umulhi(c.z, 0xCD9E8D57u);
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c;
}

// The same permutation with the round keys precomputed (k0[r], k1[r] = key
// of round r), so that each round is two wide multiplies and two 3-input xors.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys K;
    uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = k0;
        K.k1[r] = k1;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ uint4 philox(uint4 c, const PhiloxKeys &K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)c.x * 0xD2511F53u;
        const uint64_t p1 = (uint64_t)c.z * 0xCD9E8D57u;
        c = make_uint4((uint32_t)(p1 >> 32) ^ c.y ^ K.k0[r], (uint32_t)p1,
                       (uint32_t)(p0 >> 32) ^ c.w ^ K.k1[r], (uint32_t)p0);
    }
    return c;
}

// Top 24 bits of a word as a uniform in [0,1): exact in FP32 and FP64.
__device__ __forceinline__ float u24f(uint32_t x) { return (float)(x >> 8) * 0x1p-24f; }
__device__ __forceinline__ double u24d(uint32_t x) { return (double)(x >> 8) * 0x1p-24; }

// One unit of work of a persistent batch kernel: chains c0 .. c0+n-1 of
// ensemble ens.
struct BatchItem {
    uint32_t ens;
    uint32_t n;
    int64_t c0;
};

// ---------------------------------------------------------------------------
// Host-side status helpers (defined in abi.cu).
// ---------------------------------------------------------------------------
int set_error(int status, const char *fmt, ...);
int check_launch(const char *what);
// Largest dynamic shared memory a block may opt into on the current device.
int max_dynamic_smem();

// Allow a kernel the device's full opt-in shared memory.  The attribute is a
// per-function ceiling, so kernels launched with different sizes (or from
// several threads) never undercut one another.
template <class F>
inline cudaError_t allow_max_smem(F *fn)
{
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                max_dynamic_smem() - (int)fa.sharedSizeBytes);
}

}  // namespace rosen
