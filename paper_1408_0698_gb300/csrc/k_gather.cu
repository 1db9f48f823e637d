// k_gather.cu -- the host-buffer path's screen upload as a gather kernel: copies the bands of
// screen rows a frame reads (rectangles of the [L][S][S] screens, from screen_rects in api.cu)
// from pinned host memory mapped into the device's address space into the device staging
// screens, one warp per row, 16-byte loads and stores.  The rectangles are less than half the
// bytes of whole-row copies on the ELT frame; a copy engine moved them (2D copies of part rows)
// at under a third of its linear rate.
#include "internal.h"

namespace gbwfs {

namespace {
// Two warps per CTA and few registers, so that the gather's CTAs fit beside the previous frame's
// kernels on their SMs (it runs on the copy stream while they run)
constexpr int kGatherWarps = 2;
}

__global__ void __launch_bounds__(32 * kGatherWarps, 8) k_host_gather(const float4 *src, float4 *dst, int S4,
                                                                const HostRowTask *tasks, int n_tasks,
                                                                int total_rows, long long n_f4) {
    const int lane = threadIdx.x & 31;
    const int nw = gridDim.x * kGatherWarps;
    for (int g = blockIdx.x * kGatherWarps + (threadIdx.x >> 5); g < total_rows; g += nw) {
        int lo = 0, hi = n_tasks - 1;  // the last band whose first row is <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (tasks[mid].row_begin <= g) lo = mid;
            else hi = mid - 1;
        }
        const HostRowTask t = tasks[lo];
        const long long base = (t.row + (g - t.row_begin)) * (long long)S4 + t.c4_first;
        if (!guard(base >= 0 && base + t.c4_count <= n_f4, nullptr)) continue;
#pragma unroll 4
        for (int c = lane; c < t.c4_count; c += 32) dst[base + c] = src[base + c];
    }
}

cudaError_t launch_host_gather(const float *src, float *dst, int S, const HostRowTask *tasks, int n_tasks,
                               int total_rows, long long n_floats, cudaStream_t s) {
    if (total_rows <= 0 || n_tasks <= 0) return cudaSuccess;
    const int blocks = (total_rows + kGatherWarps - 1) / kGatherWarps;
    const int grid = blocks < 152 * 2 ? blocks : 152 * 2;
    k_host_gather<<<grid, 32 * kGatherWarps, 0, s>>>(reinterpret_cast<const float4 *>(src),
                                                      reinterpret_cast<float4 *>(dst), S / 4, tasks, n_tasks,
                                                      total_rows, n_floats / 4);
    return cudaGetLastError();
}

}  // namespace gbwfs
