// Displaced distance-k colouring: stencil (Eq. (9), Algorithm 2), the greedy
// walk of Algorithm 1 and a validity count.
//
// The greedy walk is sequential by definition (Sec. 4: the visit of each node
// depends on the colours of the nodes visited before it), so one CTA walks the
// visit order.  What is parallel is the gather of the neighbourhood's colours
// (Sec. 4 notes it is read-only): the CTA's threads split the stencil, OR the
// colours they see into a shared-memory bit mask, and one warp finds the first
// free colour with ballots.  Colours live in shared memory (16-bit) when the
// lattice fits, else in global memory.  Two bit masks alternate so that each
// node needs two barriers.
#include <string.h>

#include <algorithm>
#include <array>
#include <vector>

#include "pt_common.cuh"

static int build_stencil(int mu, const int *p_list, int n_p, int k, std::vector<int> &out) {
    out.clear();
    if (mu < 0 || mu > 3 || k < 0 || n_p < 1 || n_p > 64 || !p_list || k > 64) return PT_ERR_ARG;
    std::vector<std::array<int, 4>> v;
    for (int n = 0; n < n_p; ++n) {
        int p = p_list[n];
        if (p < 0 || p > 4096) return PT_ERR_ARG;
        int R = p + k;
        for (int o0 = -(mu == 0 ? R : k); o0 <= (mu == 0 ? R : k); ++o0)
            for (int o1 = -(mu == 1 ? R : k); o1 <= (mu == 1 ? R : k); ++o1)
                for (int o2 = -(mu == 2 ? R : k); o2 <= (mu == 2 ? R : k); ++o2)
                    for (int o3 = -(mu == 3 ? R : k); o3 <= (mu == 3 ? R : k); ++o3) {
                        int o[4] = {o0, o1, o2, o3};
                        if (!o0 && !o1 && !o2 && !o3) continue;
                        int dp = 0, dm = 0;
                        for (int nu = 0; nu < 4; ++nu) {
                            int c = (nu == mu) ? p : 0;
                            dp += abs(o[nu] - c);
                            dm += abs(o[nu] + c);
                        }
                        if (dp <= k || dm <= k) v.push_back({o0, o1, o2, o3});
                    }
    }
    std::sort(v.begin(), v.end());
    v.erase(std::unique(v.begin(), v.end()), v.end());
    out.reserve(v.size() * 4);
    for (auto &a : v)
        for (int nu = 0; nu < 4; ++nu) out.push_back(a[nu]);
    return PT_OK;
}

extern "C" int pt_stencil(int mu, const int *p_list, int n_p, int k, int *offsets_out, int max_offsets,
                          int *n_offsets) {
    std::vector<int> st;
    PT_CHECK_ARG(build_stencil(mu, p_list, n_p, k, st) == PT_OK && n_offsets,
                 "pt_stencil: invalid mu/p_list/k (mu in 0..3, 1 <= n_p <= 64, 0 <= p <= 4096, 0 <= k <= 64)");
    int n = (int)(st.size() / 4);
    *n_offsets = n;
    PT_CHECK_ARG(max_offsets >= n && (n == 0 || offsets_out), "pt_stencil: output holds %d rows, %d needed",
                 max_offsets, n);
    std::copy(st.begin(), st.end(), offsets_out);
    return PT_OK;
}

// site of x + o (mod D), o any integer vector
__device__ __forceinline__ int offset_site(const Geom &g, const int x[4], int4 o) {
    int c0 = (x[0] + o.x) % g.D[0]; if (c0 < 0) c0 += g.D[0];
    int c1 = (x[1] + o.y) % g.D[1]; if (c1 < 0) c1 += g.D[1];
    int c2 = (x[2] + o.z) % g.D[2]; if (c2 < 0) c2 += g.D[2];
    int c3 = (x[3] + o.w) % g.D[3]; if (c3 < 0) c3 += g.D[3];
    return c0 + g.stride[1] * c1 + g.stride[2] * c2 + g.stride[3] * c3;
}

#define PT_UNCOLOURED 0xFFFFu

template <bool SHARED_COL>
__global__ void __launch_bounds__(1024) k_colour_walk(Geom g, const int4 *__restrict__ off, int n_off,
                                                      const int *__restrict__ visit, int32_t *col, int n_words,
                                                      int *out) {
    extern __shared__ unsigned smem[];
    unsigned *used0 = smem;
    unsigned *used1 = smem + n_words;
    unsigned short *scol = reinterpret_cast<unsigned short *>(smem + 2 * n_words);
    __shared__ int s_max;
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int w = tid; w < 2 * n_words; w += nt) smem[w] = 0u;
    if (SHARED_COL)
        for (int i = tid; i < g.N; i += nt) scol[i] = PT_UNCOLOURED;
    else
        for (int i = tid; i < g.N; i += nt) col[i] = -1;
    if (tid == 0) s_max = 0;
    __syncthreads();
    for (int t = 0; t < g.N; ++t) {
        unsigned *used = (t & 1) ? used1 : used0;
        unsigned *other = (t & 1) ? used0 : used1;
        const int xs = visit[t];
        int x[4];
        site_coords(g, xs, x);
        // clear the mask of the next node while gathering this one
        for (int w = tid; w < n_words; w += nt) other[w] = 0u;
        for (int o = tid; o < n_off; o += nt) {
            int y = offset_site(g, x, off[o]);
            if (y == xs) continue;                       // x is not its own neighbour
            int c = SHARED_COL ? (int)scol[y] : col[y];
            if (SHARED_COL ? (c != (int)PT_UNCOLOURED) : (c >= 0)) atomicOr(&used[c >> 5], 1u << (c & 31));
        }
        __syncthreads();
        if (tid < 32) {
            int found = -1;
            for (int base = 0; base < n_words && found < 0; base += 32) {
                int w = base + tid;
                unsigned inv = (w < n_words) ? ~used[w] : 0u;
                unsigned bal = __ballot_sync(0xffffffffu, inv != 0u);
                if (bal) {
                    int l = __ffs(bal) - 1;
                    unsigned v = __shfl_sync(0xffffffffu, inv, l);
                    found = (base + l) * 32 + __ffs(v) - 1;
                }
            }
            if (tid == 0) {
                if (SHARED_COL) scol[xs] = (unsigned short)found;
                else col[xs] = found;
                if (found + 1 > s_max) s_max = found + 1;
            }
        }
        __syncthreads();
    }
    if (SHARED_COL)
        for (int i = tid; i < g.N; i += nt) col[i] = (int32_t)scol[i];
    if (tid == 0) out[0] = s_max;
}

__global__ void k_colour_conflicts(Geom g, const int4 *__restrict__ off, int n_off, const int32_t *__restrict__ col,
                                   unsigned long long *count) {
    __shared__ double sh[32];
    int xs = blockIdx.x * blockDim.x + threadIdx.x;
    double n = 0.0;
    if (xs < g.N) {
        int x[4];
        site_coords(g, xs, x);
        int cx = col[xs];
        for (int o = 0; o < n_off; ++o) {
            int y = offset_site(g, x, off[o]);
            if (y != xs && col[y] == cx) n += 1.0;
        }
    }
    double v[1] = {n};
    block_sum<1>(v, sh);
    if (threadIdx.x == 0 && v[0] > 0.0) atomicAdd(count, (unsigned long long)v[0]);
}

struct ColourPrep {
    int4 *d_off;
    int *d_visit;
    int *d_out;
    unsigned long long *d_count;
    int n_off;
};

static int prep(pt_ctx *c, const int dims[4], int mu, const int *p_list, int n_p, int k, int order, bool with_visit,
                ColourPrep &cp) {
    std::vector<int> st;
    PT_CHECK_ARG(build_stencil(mu, p_list, n_p, k, st) == PT_OK,
                 "colouring: invalid mu/p_list/k (mu in 0..3, 1 <= n_p <= 64, 0 <= p <= 4096, 0 <= k <= 64)");
    PT_CHECK_ARG(dims && dims[0] >= 1 && dims[1] >= 1 && dims[2] >= 1 && dims[3] >= 1, "colouring: bad dims");
    PT_CHECK_ARG(order == PT_ORDER_NATURAL || order == PT_ORDER_REDBLACK, "colouring: unknown order %d", order);
    Geom g = make_geom(dims);
    cp.n_off = (int)(st.size() / 4);
    PT_CHECK_ARG(cp.n_off < 60000, "colouring: stencil of %d offsets exceeds the 16-bit colour range", cp.n_off);
    size_t off_b = ((size_t)cp.n_off * sizeof(int4) + 255) & ~(size_t)255;
    size_t vis_b = with_visit ? (((size_t)g.N * sizeof(int) + 255) & ~(size_t)255) : 0;
    void *ws;
    int rc = pt_workspace(c, off_b + vis_b + 256, &ws);
    if (rc) return rc;
    cp.d_off = (int4 *)ws;
    cp.d_visit = (int *)((char *)ws + off_b);
    cp.d_out = (int *)((char *)ws + off_b + vis_b);
    cp.d_count = (unsigned long long *)((char *)ws + off_b + vis_b + 64);
    if (cp.n_off) PT_CUDA(cudaMemcpyAsync(cp.d_off, st.data(), st.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    if (with_visit) {
        std::vector<int> vis((size_t)g.N);
        if (order == PT_ORDER_NATURAL) {
            for (int i = 0; i < g.N; ++i) vis[i] = i;
        } else {
            size_t n = 0;
            for (int pass = 0; pass < 2; ++pass)
                for (int i = 0; i < g.N; ++i) {
                    int r = i, s = 0;
                    for (int nu = 0; nu < 4; ++nu) { s += r % dims[nu]; r /= dims[nu]; }
                    if ((s & 1) == pass) vis[n++] = i;
                }
        }
        PT_CUDA(cudaMemcpyAsync(cp.d_visit, vis.data(), vis.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
        // the host vector must outlive the copy
        PT_CUDA(cudaStreamSynchronize(c->stream));
    }
    return PT_OK;
}

extern "C" int pt_colour(pt_ctx *c, const int dims[4], int mu, const int *p_list, int n_p, int k, int order,
                         int32_t *col_dev, int *n_colours) {
    PT_CHECK_ARG(c && col_dev && n_colours, "pt_colour: NULL argument");
    PT_CUDA(cudaSetDevice(c->device));
    ColourPrep cp;
    int rc = prep(c, dims, mu, p_list, n_p, k, order, true, cp);
    if (rc) return rc;
    Geom g = make_geom(dims);
    int n_words = (cp.n_off + 2 + 31) / 32;
    size_t mask_b = 2 * (size_t)n_words * sizeof(unsigned);
    size_t shared_b = mask_b + (size_t)g.N * sizeof(unsigned short);
    int max_smem = 0;
    PT_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    max_smem -= 1024;  // static shared memory of the kernel
    if (shared_b <= (size_t)max_smem) {
        PT_CUDA(cudaFuncSetAttribute(k_colour_walk<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shared_b));
        k_colour_walk<true><<<1, 1024, shared_b, c->stream>>>(g, cp.d_off, cp.n_off, cp.d_visit, col_dev, n_words,
                                                              cp.d_out);
    } else {
        PT_CHECK_ARG(mask_b <= (size_t)max_smem, "pt_colour: stencil too large for the shared bit mask");
        PT_CUDA(cudaFuncSetAttribute(k_colour_walk<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mask_b));
        k_colour_walk<false><<<1, 1024, mask_b, c->stream>>>(g, cp.d_off, cp.n_off, cp.d_visit, col_dev, n_words,
                                                             cp.d_out);
    }
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaMemcpyAsync(c->h_flags, cp.d_out, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaStreamSynchronize(c->stream));
    *n_colours = c->h_flags[0];
    return PT_OK;
}

extern "C" int pt_colour_conflicts(pt_ctx *c, const int dims[4], int mu, const int *p_list, int n_p, int k,
                                   const int32_t *col_dev, int64_t *n_conflicts) {
    PT_CHECK_ARG(c && col_dev && n_conflicts, "pt_colour_conflicts: NULL argument");
    PT_CUDA(cudaSetDevice(c->device));
    ColourPrep cp;
    int rc = prep(c, dims, mu, p_list, n_p, k, PT_ORDER_NATURAL, false, cp);
    if (rc) return rc;
    Geom g = make_geom(dims);
    PT_CUDA(cudaMemsetAsync(cp.d_count, 0, sizeof(unsigned long long), c->stream));
    k_colour_conflicts<<<(g.N + 255) / 256, 256, 0, c->stream>>>(g, cp.d_off, cp.n_off, col_dev, cp.d_count);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    PT_CUDA(cudaMemcpyAsync(c->h_flags, cp.d_count, sizeof(unsigned long long), cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaStreamSynchronize(c->stream));
    memcpy(&h, c->h_flags, sizeof(h));
    *n_conflicts = (int64_t)h;
    return PT_OK;
}
