// abi.cu -- status strings, thread-local error text, and the exposed Philox
// stream of librosen.
#include <stdarg.h>
#include <stdio.h>

#include "common.cuh"

namespace rosen {

static thread_local char g_last_error[512] = "";

int set_error(int status, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof g_last_error, fmt, ap);
    va_end(ap);
    return status;
}

int check_launch(const char *what)
{
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "%s: %s", what, cudaGetErrorString(e));
    return ROSEN_OK;
}

int max_dynamic_smem()
{
    static thread_local int cached_dev = -1, cached = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 48 * 1024;
    if (dev != cached_dev) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
            v = 48 * 1024;
        cached = v;
        cached_dev = dev;
    }
    return cached;
}

__global__ void philox_fill_kernel(uint32_t k0, uint32_t k1, uint32_t ens, uint32_t step,
                                   uint32_t slot, uint32_t chain0, int64_t n, uint4 *out)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    out[q] = philox(make_uint4(chain0 + (uint32_t)q, ens, step, slot), k0, k1);
}

}  // namespace rosen

using namespace rosen;

extern "C" const char *rosen_status_string(int s)
{
    switch (s) {
    case ROSEN_OK: return "ROSEN_OK";
    case ROSEN_EINVAL: return "ROSEN_EINVAL";
    case ROSEN_ENOMEM: return "ROSEN_ENOMEM";
    case ROSEN_ECUDA: return "ROSEN_ECUDA";
    case ROSEN_ETIMEOUT: return "ROSEN_ETIMEOUT";
    case ROSEN_EBUSY: return "ROSEN_EBUSY";
    case ROSEN_EAGAIN: return "ROSEN_EAGAIN";
    case ROSEN_ECLOSED: return "ROSEN_ECLOSED";
    case ROSEN_ENOTFOUND: return "ROSEN_ENOTFOUND";
    default: return "ROSEN_UNKNOWN";
    }
}

extern "C" const char *rosen_last_error(void) { return g_last_error; }

extern "C" const char *rosen_version(void) { return "rosen 0.1 sm_103a"; }

extern "C" int rosen_philox(uint64_t seed, uint32_t ensemble, uint32_t step, uint32_t slot,
                            int64_t chain0, int64_t n, uint32_t *out, void *stream)
{
    if (n < 0 || chain0 < 0 || chain0 + n > (int64_t(1) << 32))
        return set_error(ROSEN_EINVAL, "rosen_philox: chain range [%lld, %lld) outside [0, 2^32)",
                         (long long)chain0, (long long)(chain0 + n));
    if (n > 0 && out == nullptr) return set_error(ROSEN_EINVAL, "rosen_philox: out is NULL");
    if (reinterpret_cast<uintptr_t>(out) & 15u)
        return set_error(ROSEN_EINVAL, "rosen_philox: out must be 16-byte aligned");
    if (n == 0) return ROSEN_OK;
    const int threads = 256;
    const int64_t blocks = (n + threads - 1) / threads;
    philox_fill_kernel<<<(unsigned)blocks, threads, 0, (cudaStream_t)stream>>>(
        (uint32_t)seed, (uint32_t)(seed >> 32), ensemble, step, slot, (uint32_t)chain0, n,
        reinterpret_cast<uint4 *>(out));
    return check_launch("rosen_philox");
}
