// tpc_find_links_noalloc: the neighbours finder and evolution of one event with all
// intermediate data in a static device array, so that the call allocates no device memory.
// The binning (A1) and neighbours (A2) kernels are the library's own; the evolution step runs
// as a variant kernel here that writes the kept links straight to the caller's arrays in input
// indices.
#include <cmath>
#include <cstring>
#include <mutex>

#include "common.cuh"
#include "../../include/tpcca.h"

namespace {

using namespace tpc;

constexpr int64_t kMaxN = TPC_NOALLOC_MAX_CLUSTERS;
constexpr int64_t kMaxR = TPC_NOALLOC_MAX_UNITS;
constexpr int64_t kSlots = kMaxN + kSlotAlign * kMaxR + 64;
// cells per unit <= 2 n + 1 (occupancy >= 0.5), each segment padded to a multiple of 4
constexpr int64_t kCells = 2 * kMaxN + (kCellAlign + 1) * kMaxR + 64;

constexpr size_t al(size_t b) { return (b + 255) & ~(size_t)255; }
constexpr size_t kOffMeta = 0;
constexpr size_t kOffDims = kOffMeta + al(kMaxR * sizeof(int4));
constexpr size_t kOffGrid = kOffDims + al(kMaxR * sizeof(int2));
constexpr size_t kOffCell = kOffGrid + al(kMaxR * sizeof(float4));
constexpr size_t kOffYz = kOffCell + al(kCells * sizeof(int32_t));
constexpr size_t kOffOrig = kOffYz + al(kSlots * sizeof(float2));
constexpr size_t kOffUp = kOffOrig + al(kSlots * sizeof(int32_t));
constexpr size_t kOffDn = kOffUp + al(kSlots * sizeof(int32_t));
constexpr size_t kOffErr = kOffDn + al(kSlots * sizeof(int32_t));
constexpr size_t kBytes = kOffErr + 256;

}  // namespace

// Scratch of tpc_find_links_noalloc.  In host code this name is only a host-side handle;
// the device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) unsigned char g_links_scratch[kBytes];

namespace {

std::mutex g_mu;                               // guards the host staging below and g_addr
void *g_addr[256];                             // device address of g_links_scratch per device
int4 g_meta[kMaxR];                            // host staging of the per-unit metadata
int2 g_dims[kMaxR];

// A3 variant: kept (reciprocal) links, written to the caller's arrays as input indices.
__global__ void __launch_bounds__(256)
k_evolve_links(const Workspace w, int64_t R, int32_t *__restrict__ up_out, int32_t *__restrict__ dn_out)
{
    for (int64_t u = blockIdx.x; u < R; u += gridDim.x) {
        const int4 m = w.meta[u];
        for (int i = threadIdx.x; i < m.y; i += blockDim.x) {
            const int cl = m.z + i;
            const int u1 = w.up_raw[cl], d1 = w.dn_raw[cl];
            const int upk = (u1 >= 0 && w.dn_raw[u1] == cl) ? u1 : -1;
            const int dnk = (d1 >= 0 && w.up_raw[d1] == cl) ? d1 : -1;
            const int me = w.orig[cl];
            up_out[me] = upk >= 0 ? w.orig[upk] : -1;
            dn_out[me] = dnk >= 0 ? w.orig[dnk] : -1;
        }
    }
}

}  // namespace

extern "C" int tpc_find_links_noalloc(tpc_tracker *tr, const float *y, const float *z, const uint8_t *row,
                                      const int32_t *counts, int64_t n, int32_t *up, int32_t *dn,
                                      int32_t *status, void *stream)
{
    TrackerInfo ti;
    if (!tracker_info(tr, &ti) || !counts || n < 0) return TPC_ERR_INVALID_ARG;
    if (n > kMaxN) return TPC_ERR_INVALID_ARG;
    if (n > 0 && (!y || !z || !row || !up || !dn)) return TPC_ERR_INVALID_ARG;
    const int nr = ti.n_rows;
    const int64_t R = (int64_t)ti.n_sectors * nr;
    if (R > kMaxR) return TPC_ERR_INVALID_ARG;
    int64_t sum = 0;
    for (int64_t u = 0; u < R; u++) {
        if (counts[u] < 0) return TPC_ERR_INVALID_ARG;
        sum += counts[u];
    }
    if (sum != n) return TPC_ERR_INVALID_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 256) return TPC_ERR_CUDA;
    cudaGetLastError();     // a launch error left over from earlier work of this thread is not this call's

    std::lock_guard<std::mutex> g(g_mu);
    if (!g_addr[dev]) {
        // once per device, with that device current
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_links_scratch) != cudaSuccess || !p) return TPC_ERR_CUDA;
        g_addr[dev] = p;
    }
    char *base = (char *)g_addr[dev];
    Workspace w;
    memset(&w, 0, sizeof w);
    w.meta = (int4 *)(base + kOffMeta);
    w.dims = (int2 *)(base + kOffDims);
    w.grid = (float4 *)(base + kOffGrid);
    w.cell = (int32_t *)(base + kOffCell);
    w.yz = (float2 *)(base + kOffYz);
    w.orig = (int32_t *)(base + kOffOrig);
    w.up_raw = (int32_t *)(base + kOffUp);
    w.dn_raw = (int32_t *)(base + kOffDn);
    w.err = (int32_t *)(base + kOffErr);
    w.pcap = kSlots;
    w.tlim = 0;
    w.ccap = kCells;
    w.rcap = kMaxR;

    // per row unit metadata, as the allocating path lays it out
    int64_t in_off = 0, s_off = 0, c_off = 0;
    int smem_need = 0, max_row = 0;
    for (int64_t u = 0; u < R; u++) {
        const int cnt = counts[u];
        const int r = (int)(u % nr);
        int ncell = (int)std::ceil((double)cnt / ti.bin_occupancy);
        if (ncell < 1) ncell = 1;
        if (ncell > kCellMax) ncell = kCellMax;
        const double wy = 2.0 * ti.row_x[r] * ti.tan_half;
        const double wz = (ti.n_sectors == 36 ? 1.0 : 2.0) * ti.z_max;
        int ny = (int)std::lround(std::sqrt(ncell * wy / wz));
        if (ny < 1) ny = 1;
        if (ny > ncell) ny = ncell;
        int nz = ncell / ny;
        if (nz < 1) nz = 1;
        g_meta[u] = make_int4((int)in_off, cnt, (int)s_off, (int)c_off);
        g_dims[u] = make_int2(ny, nz);
        if (cnt > max_row) max_row = cnt;
        in_off += cnt;
        s_off += (cnt + kSlotAlign - 1) / kSlotAlign * kSlotAlign;
        c_off += (ny * nz + 1 + kCellAlign - 1) / kCellAlign * kCellAlign;
    }
    if (s_off + 64 > kSlots || c_off + 64 > kCells) return TPC_ERR_INVALID_ARG;
    for (int64_t u = 0; u < R; u++) {
        const int r = (int)(u % nr);
        if (r == 0 || r == nr - 1) continue;
        auto rb = [](int cnt, int nc) {
            auto r16 = [](int x) { return (x + 15) & ~15; };
            return r16(cnt * 8) + r16(cnt * 4) + r16((nc + 1) * 4);
        };
        const int bytes = rb(g_meta[u + 1].y, g_dims[u + 1].x * g_dims[u + 1].y) +
                          rb(g_meta[u - 1].y, g_dims[u - 1].x * g_dims[u - 1].y);
        if (bytes > smem_need) smem_need = bytes;
    }
    const int smem = smem_need < neighbours_smem_limit() ? smem_need : neighbours_smem_limit();
    // pageable-to-device copies: the host staging is free for reuse when they return
    if (cudaMemcpyAsync(w.meta, g_meta, R * sizeof(int4), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(w.dims, g_dims, R * sizeof(int2), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(w.err, 0, 4 * sizeof(int32_t), st) != cudaSuccess)
        return TPC_ERR_CUDA;
    LaunchCfg lc;
    memset(&lc, 0, sizeof lc);
    lc.num_sms = ti.num_sms;
    lc.neighbours_block = ti.neighbours_block;
    lc.stage_rows = ti.stage_rows;
    lc.neighbours_smem_max = smem;
    lc.max_row_clusters = max_row;
    // every launch is checked on its own
    launch_ingest(*ti.dc, w, y, z, row, R, st);
    if (cudaGetLastError() != cudaSuccess) return TPC_ERR_CUDA;
    launch_neighbours(*ti.dc, w, R, smem, lc, st);
    if (cudaGetLastError() != cudaSuccess) return TPC_ERR_CUDA;
    if (R > 0) {
        int64_t grid = R < 65535 * 4 ? R : 65535 * 4;
        k_evolve_links<<<(unsigned)grid, 128, 0, st>>>(w, R, up, dn);
        if (cudaGetLastError() != cudaSuccess) return TPC_ERR_CUDA;
    }
    if (status && cudaMemcpyAsync(status, w.err, 4 * sizeof(int32_t), cudaMemcpyDeviceToDevice, st) != cudaSuccess)
        return TPC_ERR_CUDA;
    return TPC_OK;
}
