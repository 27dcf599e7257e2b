// offlattice_long.cu -- real-space growth of long chains (Guo & Baulin,
// Section 3.3.3 with the global-memory data flow the paper proposes for
// chains that do not fit in shared memory, Section 4).
//
// The rule, draws and exactness are those of rosen_offlattice_grow (same
// device code, off_chain); what changes is where a chain lives and how the
// near list of a step is found.  Every chain slot has its own region of
// device memory (positions, trace, near list) and a cell grid: the beads are
// filed by cell (side just above the list radius) in a hash table of cells,
// each heading a linked list of its beads.  A step visits the 27 cells around
// the end instead of every earlier bead, so its cost does not grow with i.
// A group of G lanes (16 or 32) grows one chain at a time and moves on to the
// next chain of its slot; as many slots run as are resident on the GPU.
#include <math.h>
#include <string.h>

#include "common.cuh"
#include "internal.cuh"
#include "offlattice_chain.cuh"

namespace rosen {
namespace {

constexpr int64_t kLongSlots = 9728;   // default slots: 152 SMs x 1024 threads / 16 lanes
constexpr size_t kLongHeader = 256;    // the chain counter, at the head of the workspace

__host__ __device__ inline size_t r16(size_t x) { return (x + 15) & ~size_t(15); }

// Cell-table entries of a chain: >= 2N (a chain fills at most N cells).
int long_log_cells(int N)
{
    int lg = 6;
    while ((int64_t(1) << lg) < 2 * (int64_t)N) ++lg;
    return lg;
}

// Device memory of one slot: hi, lo, nl, nls (N float4 each), the cell table
// (2^logH uint4), nj, njs (N int each), nb, nbs (N float each), the trace
// (N bytes); every piece starts on a 16-byte boundary.
size_t long_slot_bytes(int N, int logH)
{
    const size_t n = (size_t)N;
    return 4 * n * sizeof(float4) + ((size_t)sizeof(uint4) << logH) + 4 * r16(4 * n) + r16(n);
}

__device__ ChainLong carve_long(unsigned char *base, int N, int logH, float inv_cell, float pre2)
{
    ChainLong w;
    w.hi = reinterpret_cast<float4 *>(base);
    w.lo = w.hi + N;
    w.nl = w.lo + N;
    w.nls = w.nl + N;
    w.cells = reinterpret_cast<uint4 *>(w.nls + N);
    unsigned char *p = reinterpret_cast<unsigned char *>(w.cells + (size_t(1) << logH));
    const size_t q = r16(4 * (size_t)N);
    w.nj = reinterpret_cast<int *>(p);
    w.njs = reinterpret_cast<int *>(p + q);
    w.nb = reinterpret_cast<float *>(p + 2 * q);
    w.nbs = reinterpret_cast<float *>(p + 3 * q);
    w.tr = p + 4 * q;
    w.logH = logH;
    w.inv_cell = inv_cell;
    w.pre2 = pre2;
    return w;
}

// Each slot grows one chain at a time and takes its next chain from the
// counter *next as soon as it is done, so slots whose chains die early (most
// long hard-sphere chains) take more.
template <int G, int T, bool LJ>
__global__ void __launch_bounds__(256, 4) offlattice_long_kernel(const OffArgs a, unsigned char *ws,
                                                                 int64_t slots, size_t slot_bytes,
                                                                 int logH, float inv_cell, float pre2,
                                                                 unsigned long long *next)
{
    __shared__ float logm[kTable];
    fill_log_table(logm);
    __syncthreads();
    const Group<G> g;
    const int64_t slot = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / G;
    if (slot >= slots) return;     // whole groups leave together
    const ChainLong w = carve_long(ws + slot * slot_bytes, a.N, logH, inv_cell, pre2);
    uint32_t gen = 0;
    for (;;) {
        unsigned long long c = 0;
        if (g.gl == 0) c = atomicAdd(next, 1ull);
        c = g.bcast(c, 0);
        if (c >= (unsigned long long)a.C) break;
        off_chain<G, T, LJ>(a, (int64_t)c, w, g, logm, &gen);
    }
}

template <int G, int T, bool LJ>
int launch_long(const OffArgs &a, unsigned char *ws, size_t bytes, int logH, float inv_cell,
                float pre2, cudaStream_t s)
{
    auto kern = offlattice_long_kernel<G, T, LJ>;
    int bps = 0, dev = 0, sms = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, kern, 256, 0);
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_offlattice_grow_long: device query: %s",
                         cudaGetErrorString(e));
    const size_t slot_bytes = long_slot_bytes(a.N, logH);
    int64_t slots = bytes > kLongHeader ? (int64_t)((bytes - kLongHeader) / slot_bytes) : 0;
    const int64_t resident = (int64_t)(bps > 0 ? bps : 1) * sms * (256 / G);
    if (slots > resident) slots = resident;
    if (slots > a.C) slots = a.C;
    if (slots < 1)
        return set_error(ROSEN_ENOMEM,
                         "rosen_offlattice_grow_long: workspace of %zu bytes holds no chain slot "
                         "of %zu bytes after its %zu-byte header (N = %d)", bytes, slot_bytes,
                         kLongHeader, a.N);
    e = cudaMemsetAsync(ws, 0, kLongHeader + (size_t)slots * slot_bytes, s);
    if (e != cudaSuccess)
        return set_error(ROSEN_ECUDA, "rosen_offlattice_grow_long: clearing %lld slots of %zu bytes: %s",
                         (long long)slots, slot_bytes, cudaGetErrorString(e));
    const int64_t grid = (slots * G + 255) / 256;
    kern<<<(unsigned)grid, 256, 0, s>>>(a, ws + kLongHeader, slots, slot_bytes, logH, inv_cell, pre2,
                                       reinterpret_cast<unsigned long long *>(ws));
    return check_launch("rosen_offlattice_grow_long (kernel launch)");
}

template <int G, bool LJ>
int launch_long_g(const OffArgs &a, unsigned char *ws, size_t bytes, int logH, float inv_cell,
                  float pre2, cudaStream_t s)
{
    const int T = (a.k + G - 1) / G;
    if (T <= 1) return launch_long<G, 1, LJ>(a, ws, bytes, logH, inv_cell, pre2, s);
    if (T <= 2) return launch_long<G, 2, LJ>(a, ws, bytes, logH, inv_cell, pre2, s);
    return launch_long<G, 4, LJ>(a, ws, bytes, logH, inv_cell, pre2, s);
}

}  // namespace
}  // namespace rosen

using namespace rosen;

extern "C" size_t rosen_offlattice_long_workspace_size(int32_t N, int64_t C)
{
    if (N < 2 || N > ROSEN_OFFLATTICE_LONG_NMAX || C < 1) return 0;
    const int64_t slots = C < kLongSlots ? C : kLongSlots;
    return kLongHeader + (size_t)slots * long_slot_bytes(N, long_log_cells(N));
}

extern "C" int rosen_offlattice_grow_long(const rosen_offlattice_params *p,
                                          const rosen_offlattice_out *o, void *workspace,
                                          size_t workspace_bytes, void *stream)
{
    int st = offlattice_validate(p, o, ROSEN_OFFLATTICE_LONG_NMAX, "rosen_offlattice_grow_long");
    if (st != ROSEN_OK) return st;
    if (p->lanes_per_chain == 8)
        return set_error(ROSEN_EINVAL,
                         "rosen_offlattice_grow_long: lanes_per_chain must be 0, 16 or 32");
    if (p->C == 0) return ROSEN_OK;
    if (!workspace || (reinterpret_cast<uintptr_t>(workspace) & 15u))
        return set_error(ROSEN_EINVAL, "rosen_offlattice_grow_long: workspace must be a "
                                       "non-NULL, 16-byte aligned device pointer");
    const bool lj = p->potential == ROSEN_LJ;
    // Default lanes (measured on GB300 with the cached cell heads): hard
    // spheres take a warp per chain from N = 2048 (one cell walk per lane;
    // 71 vs 81 ms at N = 4096) and 16 lanes below (42 vs 46 ms at N = 1024);
    // Lennard-Jones the shared-memory kernel's default.
    int G = p->lanes_per_chain ? p->lanes_per_chain
                               : (lj ? offlattice_default_lanes(p->k, lj) : (p->N >= 2048 ? 32 : 16));
    if (G < 16) G = 16;
    if ((p->k + G - 1) / G > 4) G = 32;
    OffArgs a;
    offlattice_make_args(p, o, reinterpret_cast<unsigned long long *>(o->counters), &a);
    // Cell side: the list radius, plus twice the largest drift of an FP32
    // position from its exact value (4e-7 per step), plus a margin.
    const double side = sqrt((double)a.rf2) * (1.0 + 1e-6) + 2e-6 * p->N + 1e-3;
    const float inv_cell = (float)(1.0 / side);
    // Coarse-test threshold: |g|^2 from the hi words alone differs from the
    // float-float value by the lo words (<= 6e-8 |x| <= 6e-8 N per axis) and
    // FP32 rounding (< 1e-6): with d = 6e-8 N + 1e-6 and |g| <= rf + 1 the
    // difference is below 3.5 (rf + 1) d + 3 d^2 + 4e-6 rf^2; doubled.
    const double rf = sqrt((double)a.rf2);
    const double d = 6e-8 * p->N + 1e-6;
    const float pre2 =
        (float)((double)a.rf2 + 2.0 * (3.5 * (rf + 1.0) * d + 3.0 * d * d + 4e-6 * a.rf2) + 1e-6);
    const int logH = long_log_cells(p->N);
    unsigned char *ws = static_cast<unsigned char *>(workspace);
    cudaStream_t s = (cudaStream_t)stream;
    if (G == 16)
        return lj ? launch_long_g<16, true>(a, ws, workspace_bytes, logH, inv_cell, pre2, s)
                  : launch_long_g<16, false>(a, ws, workspace_bytes, logH, inv_cell, pre2, s);
    return lj ? launch_long_g<32, true>(a, ws, workspace_bytes, logH, inv_cell, pre2, s)
              : launch_long_g<32, false>(a, ws, workspace_bytes, logH, inv_cell, pre2, s);
}
