// Allocation-free variant of the colouring validity count.
//
// pt_colour_conflicts keeps its stencil table and its counter in the context's
// work space, which the library allocates with cudaMalloc.  Some callers
// cannot allow that: a host program that hands all device memory to its own
// pool allocator and forbids other allocations, a caller that must not pay
// the implicit device-wide synchronisation of cudaMalloc / cudaFree inside a
// latency-sensitive loop, or a caller running under a hard device-memory cap
// fixed at start-up.  pt_colour_conflicts_noalloc serves them: it needs no
// context, allocates nothing, and keeps its scratch in the file-scope device
// array below (PT_NOALLOC_MAX_OFFSETS stencil offsets plus one counter,
// 256 KiB + 256 B), which every device that loads the library holds until
// the process exits.
#include <string.h>

#include <algorithm>
#include <mutex>

#include "pt_common.cuh"

#define PT_NOALLOC_MAX_OFFSETS 16384
#define PT_NOALLOC_MAX_DEVICES 64

struct NoallocScratch {
    int4 off[PT_NOALLOC_MAX_OFFSETS];
    unsigned long long count;
};

static __device__ __align__(256) NoallocScratch g_noalloc_scratch;

// Host side: the device address of the array for each device (the symbol's
// name is only a host-side stand-in), and a staging table for the stencil.
static std::mutex g_noalloc_mutex;
static NoallocScratch *g_noalloc_addr[PT_NOALLOC_MAX_DEVICES];
static int4 g_noalloc_host_off[PT_NOALLOC_MAX_OFFSETS];

__device__ __forceinline__ int noalloc_offset_site(const Geom &g, const int x[4], int4 o) {
    int c0 = (x[0] + o.x) % g.D[0]; if (c0 < 0) c0 += g.D[0];
    int c1 = (x[1] + o.y) % g.D[1]; if (c1 < 0) c1 += g.D[1];
    int c2 = (x[2] + o.z) % g.D[2]; if (c2 < 0) c2 += g.D[2];
    int c3 = (x[3] + o.w) % g.D[3]; if (c3 < 0) c3 += g.D[3];
    return c0 + g.stride[1] * c1 + g.stride[2] * c2 + g.stride[3] * c3;
}

__global__ void k_conflicts_noalloc(Geom g, int n_off, const int32_t *__restrict__ col, NoallocScratch *s) {
    __shared__ double sh[32];
    const int xs = blockIdx.x * blockDim.x + threadIdx.x;
    double n = 0.0;
    if (xs < g.N) {
        int x[4];
        site_coords(g, xs, x);
        const int cx = col[xs];
        for (int o = 0; o < n_off; ++o) {
            const int y = noalloc_offset_site(g, x, s->off[o]);
            if (y != xs && col[y] == cx) n += 1.0;
        }
    }
    double v[1] = {n};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0 && v[0] > 0.0) atomicAdd(&s->count, (unsigned long long)v[0]);
}

static bool noalloc_less(const int4 &a, const int4 &b) {
    if (a.x != b.x) return a.x < b.x;
    if (a.y != b.y) return a.y < b.y;
    if (a.z != b.z) return a.z < b.z;
    return a.w < b.w;
}

static bool noalloc_same(const int4 &a, const int4 &b) { return a.x == b.x && a.y == b.y && a.z == b.z && a.w == b.w; }

// Sort the first n rows of the staging table and drop repeats; returns the
// number of distinct rows.
static int noalloc_compact(int n) {
    std::sort(g_noalloc_host_off, g_noalloc_host_off + n, noalloc_less);
    return (int)(std::unique(g_noalloc_host_off, g_noalloc_host_off + n, noalloc_same) - g_noalloc_host_off);
}

// Stencil of Eq. (8) written into the static staging table (sorted, unique).
// Repeated or overlapping displacements produce the same offset more than
// once; when the table fills up it is compacted and filling goes on, so the
// limit applies to the distinct offsets only.  Returns the number of offsets,
// or -1 if the distinct ones exceed PT_NOALLOC_MAX_OFFSETS.
static int noalloc_stencil(int mu, const int *p_list, int n_p, int k) {
    int n = 0;
    for (int q = 0; q < n_p; ++q) {
        const int p = p_list[q];
        const int R = p + k;
        const int lo[4] = {-(mu == 0 ? R : k), -(mu == 1 ? R : k), -(mu == 2 ? R : k), -(mu == 3 ? R : k)};
        int o[4];
        for (o[0] = lo[0]; o[0] <= -lo[0]; ++o[0])
            for (o[1] = lo[1]; o[1] <= -lo[1]; ++o[1])
                for (o[2] = lo[2]; o[2] <= -lo[2]; ++o[2])
                    for (o[3] = lo[3]; o[3] <= -lo[3]; ++o[3]) {
                        if (!o[0] && !o[1] && !o[2] && !o[3]) continue;
                        int dp = 0, dm = 0;
                        for (int nu = 0; nu < 4; ++nu) {
                            const int c = (nu == mu) ? p : 0;
                            dp += abs(o[nu] - c);
                            dm += abs(o[nu] + c);
                        }
                        if (dp > k && dm > k) continue;
                        if (n == PT_NOALLOC_MAX_OFFSETS) {
                            n = noalloc_compact(n);
                            if (n == PT_NOALLOC_MAX_OFFSETS) return -1;
                        }
                        g_noalloc_host_off[n++] = make_int4(o[0], o[1], o[2], o[3]);
                    }
    }
    return noalloc_compact(n);
}

extern "C" int pt_colour_conflicts_noalloc(void *stream, const int dims[4], int mu, const int *p_list, int n_p,
                                           int k, const int32_t *col_dev, int64_t *n_conflicts) {
    PT_CHECK_ARG(dims && p_list && col_dev && n_conflicts, "pt_colour_conflicts_noalloc: NULL argument");
    PT_CHECK_ARG(dims[0] >= 1 && dims[1] >= 1 && dims[2] >= 1 && dims[3] >= 1 &&
                     (int64_t)dims[0] * dims[1] * dims[2] * dims[3] < ((int64_t)1 << 31),
                 "pt_colour_conflicts_noalloc: invalid lattice dimensions");
    PT_CHECK_ARG(mu >= 0 && mu < 4 && n_p >= 1 && n_p <= 64 && k >= 0 && k <= 64,
                 "pt_colour_conflicts_noalloc: need mu in 0..3, 1 <= n_p <= 64, 0 <= k <= 64");
    for (int q = 0; q < n_p; ++q)
        PT_CHECK_ARG(p_list[q] >= 0 && p_list[q] <= 4096, "pt_colour_conflicts_noalloc: p out of range");
    int dev = 0;
    PT_CUDA(cudaGetDevice(&dev));
    PT_CHECK_ARG(dev >= 0 && dev < PT_NOALLOC_MAX_DEVICES, "pt_colour_conflicts_noalloc: device %d unsupported", dev);
    cudaStream_t st = (cudaStream_t)stream;

    // One call at a time per process: the scratch array and the host staging
    // table are shared, and every call finishes on the GPU before it returns.
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_addr[dev]) {
        // set-up, once per device, with that device current
        void *p = nullptr;
        PT_CUDA(cudaGetSymbolAddress(&p, g_noalloc_scratch));
        g_noalloc_addr[dev] = (NoallocScratch *)p;
    }
    NoallocScratch *s = g_noalloc_addr[dev];
    const int n_off = noalloc_stencil(mu, p_list, n_p, k);
    PT_CHECK_ARG(n_off >= 0, "pt_colour_conflicts_noalloc: stencil exceeds the %d-offset scratch limit",
                 PT_NOALLOC_MAX_OFFSETS);
    const Geom g = make_geom(dims);
    unsigned long long h_count = 0;
    if (n_off > 0)
        PT_CUDA(cudaMemcpyAsync(s->off, g_noalloc_host_off, (size_t)n_off * sizeof(int4), cudaMemcpyHostToDevice, st));
    // the counter keeps the previous call's value: clear it
    PT_CUDA(cudaMemsetAsync(&s->count, 0, sizeof(unsigned long long), st));
    k_conflicts_noalloc<<<(g.N + 255) / 256, 256, 0, st>>>(g, n_off, col_dev, s);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaMemcpyAsync(&h_count, &s->count, sizeof(h_count), cudaMemcpyDeviceToHost, st));
    PT_CUDA(cudaStreamSynchronize(st));
    *n_conflicts = (int64_t)h_count;
    return PT_OK;
}
