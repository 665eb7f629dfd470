// Displaced distance-k colouring: stencil (Eq. (8), Algorithm 2), the greedy
// walk of Algorithm 1 and a validity count.
//
// The greedy walk is sequential by definition (Sec. 4: the visit of each node
// depends on the colours of the nodes visited before it), so one CTA walks the
// visit order.  What is parallel is the gather of the neighbourhood's colours
// (Sec. 4 notes it is read-only): the CTA's threads split the stencil, stamp
// the colours they see into a shared-memory table, and search it for the
// first free colour.  Lattices whose 16-bit colours fit in shared memory keep
// them there (k_colour_walk); larger ones keep them in an extended array in
// global memory, read through L1, with two nodes in flight per barrier
// (k_colour_walk_ext).
#include <limits.h>
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
#define PT_WALK_U 16

// Walk offsets: every stencil offset reduced to [0, D_mu) per dimension and
// packed as two 16-bit pairs (o0 | o1 << 16, o2 | o3 << 16).  Offsets equal
// modulo the lattice reach the same node and are merged; the one equal to 0
// (x itself, excluded from N(x, p, k)) is dropped.  The neighbour's
// coordinate is then x + o with at most one subtraction of D.
__device__ __forceinline__ int walk_site(const Geom &g, const int x[4], uint2 o) {
    int c0 = x[0] + (int)(o.x & 0xffffu); c0 -= (c0 >= g.D[0]) ? g.D[0] : 0;
    int c1 = x[1] + (int)(o.x >> 16);     c1 -= (c1 >= g.D[1]) ? g.D[1] : 0;
    int c2 = x[2] + (int)(o.y & 0xffffu); c2 -= (c2 >= g.D[2]) ? g.D[2] : 0;
    int c3 = x[3] + (int)(o.y >> 16);     c3 -= (c3 >= g.D[3]) ? g.D[3] : 0;
    return c0 + g.stride[1] * c1 + g.stride[2] * c2 + g.stride[3] * c3;
}

// One node per step, three phases and two barriers per node:
//   gather  every thread takes its share of the offsets, loads the colours of
//           the neighbours (PT_WALK_U loads in flight before any is used) and
//           stamps each colour seen: stamp[c] = step (a plain store; threads
//           that see the same colour write the same value);
//   search  the first colour c in [0, m] without this step's stamp, m the
//           colours used so far: each thread checks its stride of c, warps
//           reduce, one shared atomicMin per warp;
//   commit  every thread reads the winner; thread 0 stores it.
// Stamps grow with the step, so they are never cleared.  The node coloured in
// one step may be a neighbour of the next node before its colour store is
// visible to the other threads, so every thread keeps (node, colour) of the
// previous step and uses it in the next gather.  Shared memory: the stamps
// (n_stamp ints), then (SHARED_OFF) the packed offsets, then (SHARED_COL) the
// 16-bit colours of all N nodes.  NESTED: a node only sees the neighbours
// with its own parent colour (parent[], the coarser colouring), and the
// colours found are local to each parent class.
template <bool SHARED_COL, bool SHARED_OFF, bool NESTED>
__global__ void __launch_bounds__(1024, 1) k_colour_walk(Geom g, const uint2 *__restrict__ off_g, int n_off,
                                                      const int *__restrict__ visit, int32_t *col, int n_stamp,
                                                      int *out, const int32_t *__restrict__ parent) {
    extern __shared__ int smem_i[];
    int *stamp = smem_i;
    uint2 *soff = reinterpret_cast<uint2 *>(smem_i + ((n_stamp + 1) & ~1));
    unsigned short *scol = reinterpret_cast<unsigned short *>(soff + (SHARED_OFF ? n_off : 0));
    const uint2 *off = SHARED_OFF ? soff : off_g;
    __shared__ int s_found[2];
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int c = tid; c < n_stamp; c += nt) stamp[c] = 0;
    if (SHARED_OFF)
        for (int o = tid; o < n_off; o += nt) soff[o] = off_g[o];
    if (SHARED_COL)
        for (int i = tid; i < g.N; i += nt) scol[i] = PT_UNCOLOURED;
    else
        for (int i = tid; i < g.N; i += nt) col[i] = -1;
    if (tid == 0) s_found[0] = s_found[1] = INT_MAX;
    __syncthreads();
    int m = 0;                       // colours used so far (the same in every thread)
    int prev_x = -1, prev_c = -1;    // node and colour of the previous step
    int xs_next = visit[0];
    for (int t = 0; t < g.N; ++t) {
        const int step = t + 1;
        const int xs = xs_next;
        if (t + 1 < g.N) xs_next = visit[t + 1];          // in flight during this node's gather
        int x[4];
        site_coords(g, xs, x);
        const int px = NESTED ? parent[xs] : 0;
        for (int base = tid; base < n_off; base += nt * PT_WALK_U) {
            int cv[PT_WALK_U];
#pragma unroll
            for (int u = 0; u < PT_WALK_U; ++u) {
                const int o = base + u * nt;
                cv[u] = -1;
                if (o < n_off) {
                    const int y = walk_site(g, x, off[o]);
                    int c = SHARED_COL ? (int)scol[y] : col[y];
                    if (SHARED_COL && c == (int)PT_UNCOLOURED) c = -1;
                    cv[u] = (y == prev_x) ? prev_c : c;
                    if (NESTED && parent[y] != px) cv[u] = -1;
                }
            }
#pragma unroll
            for (int u = 0; u < PT_WALK_U; ++u)
                if (cv[u] >= 0) stamp[cv[u]] = step;
        }
        __syncthreads();
        int best = INT_MAX;
        for (int c = tid; c <= m; c += nt)
            if (stamp[c] != step) { best = c; break; }
        best = __reduce_min_sync(0xffffffffu, best);
        if ((tid & 31) == 0 && best != INT_MAX) atomicMin(&s_found[t & 1], best);
        __syncthreads();
        const int found = s_found[t & 1];
        if (tid == 0) {
            if (SHARED_COL) scol[xs] = (unsigned short)found;
            else col[xs] = found;
            s_found[(t + 1) & 1] = INT_MAX;               // read by nobody before the next step's first barrier
        }
        if (found + 1 > m) m = found + 1;
        prev_x = xs;
        prev_c = found;
    }
    __syncthreads();
    if (SHARED_COL)
        for (int i = tid; i < g.N; i += nt) col[i] = (int32_t)scol[i];
    if (tid == 0) out[0] = m;
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

// Walk with the colours in an extended array: the lattice plus halos wide
// enough that every neighbour x + o is a plain index offset,
// colext[b(x) + delta_o], with no wrap arithmetic; a node's colour is written
// to each of its periodic images in the array (at most two per dimension).
//
// One barrier per node, two nodes in flight: between two barriers the CTA
// commits the colour of node t-1 (found by the previous search), gathers the
// neighbourhood of node t+1 into one stamp buffer and searches node t's
// (gathered before the previous barrier) in the other.  A gather cannot see
// the colours of the two nodes before it (one not yet found, one being
// written), so the search of node t skips those two colours itself when the
// nodes are neighbours of t: the L1 distance to the nearer displaced image
// (Eq. (8)), tested one node ahead by two threads and kept in shared memory.
// Each thread holds its U offsets' deltas in registers for the whole walk
// and issues all its loads of a gather before using any of them; both stamp
// buffers live in shared memory, the colours come through L1.
#define PT_EXT_NT 1024
struct ExtGeom {
    int lo[4];      // smallest offset coordinate per dimension (<= 0)
    int E[4];       // extended sides
    int ES[4];      // extended strides
    int mu, k, n_p;
    int p[64];      // displacements reduced mod D_mu
};

// distance to the nearest multiple of D, for |v| < 2D
__device__ __forceinline__ int dist_mod(int v, int D) {
    v += (v < 0) ? D : 0;
    v += (v < 0) ? D : 0;
    v -= (v >= D) ? D : 0;
    return min(v, D - v);
}

// is node a (coordinates) in N(b, p, k) for some p of the list?
__device__ __forceinline__ bool ext_neighbour(const Geom &g, const ExtGeom &eg, const int a[4], const int b[4]) {
    int rest = 0, dm = 0, Dm = 1;
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) {
        const int dd = a[nu] - b[nu];
        if (nu == eg.mu) { dm = dd; Dm = g.D[nu]; }
        else rest += dist_mod(dd, g.D[nu]);
    }
    int best = INT_MAX;
    for (int n = 0; n < eg.n_p; ++n) best = min(best, min(dist_mod(dm - eg.p[n], Dm), dist_mod(dm + eg.p[n], Dm)));
    return rest + best <= eg.k;
}

__device__ __forceinline__ int ext_base(const ExtGeom &eg, const int x[4]) {
    return (x[0] - eg.lo[0]) + eg.ES[1] * (x[1] - eg.lo[1]) + eg.ES[2] * (x[2] - eg.lo[2]) + eg.ES[3] * (x[3] - eg.lo[3]);
}

// stamp[c] = value for the colour of every neighbour that has one; this
// thread's n_mine offsets are dlt[0..n_mine)
template <int U>
__device__ __forceinline__ void ext_gather(const int (&dlt)[U], int n_mine, const unsigned short *colext, int b,
                                           int *stamp, int value) {
    unsigned short cv[U];
#pragma unroll
    for (int u = 0; u < U; ++u) cv[u] = (u < n_mine) ? colext[b + dlt[u]] : (unsigned short)PT_UNCOLOURED;
#pragma unroll
    for (int u = 0; u < U; ++u)
        if (cv[u] != PT_UNCOLOURED) stamp[cv[u]] = value;
}

template <int U>
__global__ void __launch_bounds__(PT_EXT_NT, 1) k_colour_walk_ext(Geom g, ExtGeom eg, const int *__restrict__ delta,
                                                                  int n_off, const int *__restrict__ visit,
                                                                  unsigned short *colext, int32_t *col,
                                                                  int n_stamp, int *out) {
    extern __shared__ int sm_ext[];  // two stamp buffers of n_stamp ints
    __shared__ int s_found[3];       // search results, one slot per node mod 3
    __shared__ int s_nb[4];          // [parity of node][0: node - 1 is a neighbour, 1: node - 2 is]
    const int tid = threadIdx.x;
    for (int c = tid; c < 2 * n_stamp; c += PT_EXT_NT) sm_ext[c] = 0;
    int dlt[U];                      // this thread's offsets: tid, tid + NT, ...
#pragma unroll
    for (int u = 0; u < U; ++u) dlt[u] = (tid + u * PT_EXT_NT < n_off) ? delta[tid + u * PT_EXT_NT] : 0;
    const int n_mine = (n_off > tid) ? (n_off - tid + PT_EXT_NT - 1) / PT_EXT_NT : 0;
    if (tid < 3) s_found[tid] = INT_MAX;
    if (tid < 4) s_nb[tid] = 0;
    __syncthreads();
    // node history: x0 = node t, x1 = t - 1, x2 = t - 2, xn = t + 1 (coordinates and index)
    int x0[4], x1[4], x2[4], xn[4];
    int i0 = visit[0], i1 = -1, i2 = -1, in_ = -1;
    site_coords(g, i0, x0);
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) x1[nu] = x2[nu] = xn[nu] = 0;
    int f1 = -1, f2 = -1;            // colours of nodes t - 1 and t - 2
    int m = 0;                       // colours used by nodes before t
    int i_next = (g.N > 1) ? visit[1] : 0;
    ext_gather<U>(dlt, n_mine, colext, ext_base(eg, x0), sm_ext, 1);
    __syncthreads();
    for (int t = 0; t < g.N; ++t) {
        // commit node t - 1, whose colour the previous search found
        if (t >= 1) {
            const int f = s_found[(t - 1) % 3];
            if (tid < 16) {
                int e = 0, ok = 1;
#pragma unroll
                for (int nu = 0; nu < 4; ++nu) {
                    int ev = x1[nu] - eg.lo[nu];                 // in [0, 2D): one reduction
                    ev -= (ev >= g.D[nu]) ? g.D[nu] : 0;
                    ev += ((tid >> nu) & 1) * g.D[nu];
                    ok &= ev < eg.E[nu];
                    e += ev * eg.ES[nu];
                }
                if (ok) colext[e] = (unsigned short)f;
            }
            if (tid == 0) col[i1] = f;
            f2 = f1;
            f1 = f;
            if (f + 1 > m) m = f + 1;
        }
        if (tid == 0) s_found[(t + 1) % 3] = INT_MAX;      // last read before the previous barrier
        // gather node t + 1
        if (t + 1 < g.N) {
            in_ = i_next;
            if (t + 2 < g.N) i_next = visit[t + 2];
            site_coords(g, in_, xn);
            // for the search of node t + 1: are nodes t and t - 1 its neighbours?
            if (tid == 32) s_nb[2 * ((t + 1) & 1)] = ext_neighbour(g, eg, x0, xn);
            if (tid == 64) s_nb[2 * ((t + 1) & 1) + 1] = (i1 >= 0) && ext_neighbour(g, eg, x1, xn);
            ext_gather<U>(dlt, n_mine, colext, ext_base(eg, xn), sm_ext + ((t + 1) & 1) * n_stamp, t + 2);
        }
        // search node t: smallest colour in [0, m] not stamped and not held by a neighbouring t-1 or t-2
        const int skip1 = s_nb[2 * (t & 1)] ? f1 : -1;
        const int skip2 = s_nb[2 * (t & 1) + 1] ? f2 : -1;
        const int *st = sm_ext + (t & 1) * n_stamp;
        int best = INT_MAX;
        for (int c = tid; c <= m; c += PT_EXT_NT)
            if (st[c] != t + 1 && c != skip1 && c != skip2) { best = c; break; }
        best = __reduce_min_sync(0xffffffffu, best);
        if ((tid & 31) == 0 && best != INT_MAX) atomicMin(&s_found[t % 3], best);
        __syncthreads();
        // shift the history
        i2 = i1; i1 = i0; i0 = in_;
#pragma unroll
        for (int nu = 0; nu < 4; ++nu) { x2[nu] = x1[nu]; x1[nu] = x0[nu]; x0[nu] = xn[nu]; }
    }
    if (tid == 0) {
        const int f = s_found[(g.N - 1) % 3];
        col[i1] = f;
        out[0] = (f + 1 > m) ? f + 1 : m;
    }
}

// Offsets of the walk: reduced modulo the lattice, merged, x itself dropped,
// packed (see walk_site).  Sides are below 65536 (PT_CHECK in the caller).
static std::vector<uint2> walk_offsets(const std::vector<int> &st, const int dims[4]) {
    std::vector<uint64_t> keys;
    keys.reserve(st.size() / 4);
    for (size_t i = 0; i < st.size(); i += 4) {
        uint64_t key = 0;
        bool zero = true;
        for (int nu = 0; nu < 4; ++nu) {
            int c = st[i + nu] % dims[nu];
            if (c < 0) c += dims[nu];
            zero = zero && c == 0;
            key |= (uint64_t)c << (16 * nu);
        }
        if (!zero) keys.push_back(key);
    }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
    std::vector<uint2> out(keys.size());
    for (size_t i = 0; i < keys.size(); ++i) out[i] = make_uint2((unsigned)keys[i], (unsigned)(keys[i] >> 32));
    return out;
}

// The greedy walk of pt_colour (parent == NULL) and of pt_colour_nested (the
// local colours of each parent class).  *m receives the colour count; the
// visit order stays in the work space (ColourPrep) for the caller.
static int colour_walk(pt_ctx *c, const int dims[4], int mu, const int *p_list, int n_p, int k, int order,
                       const int32_t *parent, int32_t *col_dev, int *n_colours, ColourPrep &cp) {
    PT_CHECK_ARG(c && col_dev && n_colours, "pt_colour: NULL argument");
    PT_CHECK_ARG(dims && dims[0] < 65536 && dims[1] < 65536 && dims[2] < 65536 && dims[3] < 65536,
                 "pt_colour: lattice sides must be below 65536");
    PT_CUDA(cudaSetDevice(c->device));
    int rc = prep(c, dims, mu, p_list, n_p, k, order, true, cp);
    if (rc) return rc;
    Geom g = make_geom(dims);
    std::vector<int> st;
    build_stencil(mu, p_list, n_p, k, st);
    std::vector<uint2> wo = walk_offsets(st, dims);
    const int n_off = (int)wo.size();
    // the packed offsets take the place of the int4 stencil in the workspace (8 <= 16 bytes per row)
    uint2 *d_off = reinterpret_cast<uint2 *>(cp.d_off);
    if (n_off) PT_CUDA(cudaMemcpyAsync(d_off, wo.data(), wo.size() * sizeof(uint2), cudaMemcpyHostToDevice, c->stream));
    // a node's colour never exceeds its number of neighbours: stamps for 0..n_off
    const int n_stamp = n_off + 2;
    const size_t stamp_b = (size_t)((n_stamp + 1) & ~1) * sizeof(int);
    size_t off_b = (size_t)n_off * sizeof(uint2);
    size_t col_b = (size_t)g.N * sizeof(unsigned short);
    int max_smem = 0;
    PT_CUDA(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
    max_smem -= 1024;  // static shared memory of the kernel
    PT_CHECK_ARG(stamp_b <= (size_t)max_smem, "pt_colour: stencil too large for the shared colour stamps");
    const bool sh_col = stamp_b + col_b <= (size_t)max_smem;
    const bool sh_off = stamp_b + off_b + (sh_col ? col_b : 0) <= (size_t)max_smem;
    size_t shared_b = stamp_b + (sh_off ? off_b : 0) + (sh_col ? col_b : 0);
    // large lattices: the extended-array walk (two stamp buffers in shared memory, deltas in registers)
    const size_t ext_smem = (size_t)(2 * n_stamp) * sizeof(int);
    if (!parent && !sh_col && ext_smem <= (size_t)max_smem && n_p <= 64 && n_off <= PT_EXT_NT * 24) {
        ExtGeom eg;
        eg.mu = mu;
        eg.k = k;
        eg.n_p = n_p;
        for (int n = 0; n < n_p; ++n) eg.p[n] = p_list[n] % dims[mu];
        // per dimension: signed offsets if the largest minimal image R fits (2R + 1 <= D), else [0, D)
        int sgn[4];
        long E = 1;
        for (int nu = 0; nu < 4; ++nu) {
            int R = 0, hi = 0;
            for (const uint2 &o : wo) {
                const unsigned w = (nu < 2) ? o.x : o.y;
                const int r = (int)((nu & 1) ? (w >> 16) : (w & 0xffffu));
                R = std::max(R, std::min(r, dims[nu] - r));
                hi = std::max(hi, r);
            }
            sgn[nu] = 2 * R + 1 <= dims[nu];
            eg.lo[nu] = sgn[nu] ? -R : 0;
            eg.E[nu] = dims[nu] + (sgn[nu] ? 2 * R : hi);
            eg.ES[nu] = (int)E;
            E *= eg.E[nu];
        }
        PT_CHECK_ARG(E < (1L << 31), "pt_colour: extended lattice too large");
        std::vector<int> delta(n_off);
        for (int i = 0; i < n_off; ++i) {
            long dl = 0;
            for (int nu = 0; nu < 4; ++nu) {
                const unsigned w = (nu < 2) ? wo[i].x : wo[i].y;
                const int r = (int)((nu & 1) ? (w >> 16) : (w & 0xffffu));
                const int o = (sgn[nu] && r > dims[nu] - r) ? r - dims[nu] : r;
                dl += (long)o * eg.ES[nu];
            }
            delta[i] = (int)dl;
        }
        unsigned short *d_ext = nullptr;
        int *d_delta = nullptr;
        PT_CUDA(cudaMallocAsync((void **)&d_ext, (size_t)E * sizeof(unsigned short), c->stream));
        PT_CUDA(cudaMallocAsync((void **)&d_delta, (size_t)std::max(n_off, 1) * sizeof(int), c->stream));
        PT_CUDA(cudaMemsetAsync(d_ext, 0xff, (size_t)E * sizeof(unsigned short), c->stream));
        if (n_off)
            PT_CUDA(cudaMemcpyAsync(d_delta, delta.data(), delta.size() * sizeof(int), cudaMemcpyHostToDevice,
                                    c->stream));
#define PT_EXT(U)                                                                                                \
    do {                                                                                                         \
        PT_CUDA(cudaFuncSetAttribute(k_colour_walk_ext<U>, cudaFuncAttributeMaxDynamicSharedMemorySize,          \
                                     (int)ext_smem));                                                            \
        k_colour_walk_ext<U><<<1, PT_EXT_NT, ext_smem, c->stream>>>(g, eg, d_delta, n_off, cp.d_visit, d_ext,    \
                                                                    col_dev, n_stamp, cp.d_out);                 \
    } while (0)
        if (n_off <= PT_EXT_NT * 4) PT_EXT(4);
        else if (n_off <= PT_EXT_NT * 8) PT_EXT(8);
        else if (n_off <= PT_EXT_NT * 12) PT_EXT(12);
        else if (n_off <= PT_EXT_NT * 16) PT_EXT(16);
        else if (n_off <= PT_EXT_NT * 20) PT_EXT(20);
        else PT_EXT(24);
#undef PT_EXT
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        PT_CUDA(cudaFreeAsync(d_ext, c->stream));
        PT_CUDA(cudaFreeAsync(d_delta, c->stream));
        PT_CUDA(cudaMemcpyAsync(c->h_flags, cp.d_out, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        PT_CUDA(cudaStreamSynchronize(c->stream));
        *n_colours = c->h_flags[0];
        return PT_OK;
    }
#define PT_WALK(SC, SO, NE)                                                                                      \
    do {                                                                                                         \
        PT_CUDA(cudaFuncSetAttribute(k_colour_walk<SC, SO, NE>, cudaFuncAttributeMaxDynamicSharedMemorySize,      \
                                     (int)shared_b));                                                            \
        k_colour_walk<SC, SO, NE><<<1, 1024, shared_b, c->stream>>>(g, d_off, n_off, cp.d_visit, col_dev,        \
                                                                    n_stamp, cp.d_out, parent);                  \
    } while (0)
    if (parent) {
        if (sh_col && sh_off) PT_WALK(true, true, true);
        else if (sh_col) PT_WALK(true, false, true);
        else if (sh_off) PT_WALK(false, true, true);
        else PT_WALK(false, false, true);
    } else {
        if (sh_col && sh_off) PT_WALK(true, true, false);
        else if (sh_col) PT_WALK(true, false, false);
        else if (sh_off) PT_WALK(false, true, false);
        else PT_WALK(false, false, false);
    }
#undef PT_WALK
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaMemcpyAsync(c->h_flags, cp.d_out, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaStreamSynchronize(c->stream));
    *n_colours = c->h_flags[0];
    return PT_OK;
}

extern "C" int pt_colour(pt_ctx *c, const int dims[4], int mu, const int *p_list, int n_p, int k, int order,
                         int32_t *col_dev, int *n_colours) {
    ColourPrep cp;
    return colour_walk(c, dims, mu, p_list, n_p, k, order, nullptr, col_dev, n_colours, cp);
}

// ------------------------------------------------------------ nested colouring
// The colour of a node is the pair (parent colour, local colour); pairs are
// numbered in the order the walk first meets them: each pair's first visit
// rank (atomicMin over its nodes), then its position among the pairs sorted
// by that rank, then the number written to every node.

#define PT_PAIR_UNSET 0x7f7f7f7f      // bytes 0x7f: larger than any visit rank

__global__ void k_visit_rank(int N, const int *__restrict__ visit, int *rank) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < N; t += gridDim.x * blockDim.x) rank[visit[t]] = t;
}

__global__ void k_pair_first(int N, const int32_t *__restrict__ parent, int n_parent, const int32_t *__restrict__ local,
                             int m_local, const int *__restrict__ rank, int *first, int *bad) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const int pa = parent[x], lo = local[x];
        if (pa < 0 || pa >= n_parent || lo < 0 || lo >= m_local) { atomicOr(bad, 1); continue; }
        atomicMin(&first[(size_t)pa * m_local + lo], rank[x]);
    }
}

// id of a used pair = number of used pairs met earlier; *n_used counts them
__global__ void k_pair_ids(int K, const int *__restrict__ first, int *id, int *n_used) {
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < K; q += gridDim.x * blockDim.x) {
        const int f = first[q];
        if (f == PT_PAIR_UNSET) { id[q] = -1; continue; }
        int n = 0;
        for (int r = 0; r < K; ++r) n += first[r] < f;
        id[q] = n;
        atomicAdd(n_used, 1);
    }
}

__global__ void k_pair_assign(int N, const int32_t *__restrict__ parent, int m_local, const int *__restrict__ id,
                              int32_t *col) {
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x)
        col[x] = id[(size_t)parent[x] * m_local + col[x]];
}

extern "C" int pt_colour_nested(pt_ctx *c, const int dims[4], int mu, const int *p_list, int n_p, int k, int order,
                                const int32_t *parent_dev, int n_parent, int32_t *col_dev, int *n_colours) {
    PT_CHECK_ARG(c && parent_dev && col_dev && n_colours, "pt_colour_nested: NULL argument");
    PT_CHECK_ARG(n_parent >= 1, "pt_colour_nested: n_parent must be at least 1");
    ColourPrep cp;
    int m_local = 0;
    int rc = colour_walk(c, dims, mu, p_list, n_p, k, order, parent_dev, col_dev, &m_local, cp);
    if (rc) return rc;
    Geom g = make_geom(dims);
    const long K = (long)n_parent * m_local;
    PT_CHECK_ARG(g.N < PT_PAIR_UNSET, "pt_colour_nested: lattice too large");
    PT_CHECK_ARG(K <= (1L << 24), "pt_colour_nested: %ld (parent, local) pairs exceed the table", K);
    // work space after the visit order: rank [N], first [K], id [K], two flags
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t rank_b = al((size_t)g.N * sizeof(int)), k_b = al((size_t)K * sizeof(int));
    int32_t *tmp = nullptr;
    PT_CUDA(cudaMallocAsync((void **)&tmp, rank_b + 2 * k_b + 256, c->stream));
    int *rank = (int *)tmp, *first = (int *)((char *)tmp + rank_b), *id = (int *)((char *)tmp + rank_b + k_b);
    int *flags = (int *)((char *)tmp + rank_b + 2 * k_b);
    PT_CUDA(cudaMemsetAsync(first, 0x7f, (size_t)K * sizeof(int), c->stream));   // PT_PAIR_UNSET
    PT_CUDA(cudaMemsetAsync(flags, 0, 2 * sizeof(int), c->stream));
    const int blocks = (int)std::min<long>(((long)g.N + 255) / 256, 16L * c->num_sms);
    const int kblocks = (int)std::min<long>((K + 255) / 256, 16L * c->num_sms);
    k_visit_rank<<<blocks, 256, 0, c->stream>>>(g.N, cp.d_visit, rank);
    k_pair_first<<<blocks, 256, 0, c->stream>>>(g.N, parent_dev, n_parent, col_dev, m_local, rank, first, flags);
    pt_kernel_launch_count += 2;
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaMemcpyAsync(c->h_flags, flags, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaStreamSynchronize(c->stream));
    if (c->h_flags[0]) {
        cudaFreeAsync(tmp, c->stream);
        PT_CHECK_ARG(false, "pt_colour_nested: parent colours must lie in [0, n_parent)");
    }
    k_pair_ids<<<kblocks, 256, 0, c->stream>>>((int)K, first, id, flags + 1);
    k_pair_assign<<<blocks, 256, 0, c->stream>>>(g.N, parent_dev, m_local, id, col_dev);
    pt_kernel_launch_count += 2;
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaMemcpyAsync(c->h_flags, flags + 1, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaFreeAsync(tmp, c->stream));
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

// ------------------------------------------------------------------ tiles
// Tile policy of Sec. 3.5: every side at least 2k + 1, the displaced side at
// least 2(p_max + k) + 1, each side the smallest divisor of the lattice side
// at or above that minimum (a power of two for power-of-two lattices), else
// the lattice side itself.

static int tile_side(int D, int need) {
    for (int t = 1; t <= D; ++t)
        if (D % t == 0 && t >= need) return t;
    return D;
}

extern "C" int pt_tile_dims(const int dims[4], int mu, const int *p_list, int n_p, int k, int tile_out[4]) {
    PT_CHECK_ARG(dims && p_list && tile_out && n_p >= 1 && n_p <= 64 && mu >= 0 && mu <= 3 && k >= 0 && k <= 64,
                 "pt_tile_dims: invalid arguments");
    int pmax = 0;
    for (int n = 0; n < n_p; ++n) {
        PT_CHECK_ARG(p_list[n] >= 0 && p_list[n] <= 4096, "pt_tile_dims: displacement %d out of range", p_list[n]);
        pmax = std::max(pmax, p_list[n]);
    }
    for (int nu = 0; nu < 4; ++nu) {
        PT_CHECK_ARG(dims[nu] >= 1, "pt_tile_dims: bad lattice side");
        int need = (nu == mu) ? 2 * (pmax + k) + 1 : 2 * k + 1;
        tile_out[nu] = tile_side(dims[nu], need);
    }
    return PT_OK;
}

__global__ void k_tile_replicate(Geom g, Geom tg, const int32_t *__restrict__ tcol, int32_t *__restrict__ col) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
        int x[4];
        site_coords(g, i, x);
        int j = (x[0] % tg.D[0]) + tg.stride[1] * (x[1] % tg.D[1]) + tg.stride[2] * (x[2] % tg.D[2]) +
                tg.stride[3] * (x[3] % tg.D[3]);
        col[i] = tcol[j];
    }
}

extern "C" int pt_tile_replicate(pt_ctx *c, const int tile_dims[4], const int32_t *tile_col_dev, const int dims[4],
                                 int32_t *col_dev) {
    PT_CHECK_ARG(c && tile_dims && tile_col_dev && dims && col_dev, "pt_tile_replicate: NULL argument");
    for (int nu = 0; nu < 4; ++nu)
        PT_CHECK_ARG(tile_dims[nu] >= 1 && dims[nu] >= 1 && dims[nu] % tile_dims[nu] == 0,
                     "pt_tile_replicate: tile side %d does not divide lattice side %d", tile_dims[nu], dims[nu]);
    Geom g = make_geom(dims), tg = make_geom(tile_dims);
    PT_CHECK_ARG(tile_col_dev + tg.N <= col_dev || col_dev + g.N <= tile_col_dev,
                 "pt_tile_replicate: tile and lattice colourings overlap");
    PT_CUDA(cudaSetDevice(c->device));
    int blocks = (int)std::min<long>(((long)g.N + 255) / 256, 16L * c->num_sms);
    k_tile_replicate<<<blocks, 256, 0, c->stream>>>(g, tg, tile_col_dev, col_dev);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}

extern "C" int pt_colour_tiled(pt_ctx *c, const int dims[4], int mu, const int *p_list, int n_p, int k, int order,
                               int32_t *col_dev, int *n_colours, int tile_out[4]) {
    PT_CHECK_ARG(c && dims && col_dev && n_colours && tile_out, "pt_colour_tiled: NULL argument");
    int rc = pt_tile_dims(dims, mu, p_list, n_p, k, tile_out);
    if (rc) return rc;
    if (tile_out[0] == dims[0] && tile_out[1] == dims[1] && tile_out[2] == dims[2] && tile_out[3] == dims[3])
        return pt_colour(c, dims, mu, p_list, n_p, k, order, col_dev, n_colours);
    PT_CUDA(cudaSetDevice(c->device));
    size_t nt = (size_t)tile_out[0] * tile_out[1] * tile_out[2] * tile_out[3];
    int32_t *tcol = nullptr;
    PT_CUDA(cudaMallocAsync((void **)&tcol, nt * sizeof(int32_t), c->stream));
    rc = pt_colour(c, tile_out, mu, p_list, n_p, k, order, tcol, n_colours);
    if (rc == PT_OK) rc = pt_tile_replicate(c, tile_out, tcol, dims, col_dev);
    cudaFreeAsync(tcol, c->stream);
    if (rc == PT_OK) PT_CUDA(cudaStreamSynchronize(c->stream));
    return rc;
}

// -------------------------------------------------------------- clearance
// Table 5 (Sec. 4.3): for displacement p and distance k, the shell S(p, k) is
// the set of nodes y != x whose distance to the nearer of x + p e_mu and
// x - p e_mu is exactly k; the statistic is the number of (x, y in S_x) pairs
// with equal colours.  On the torus the shell's offsets, reduced mod D, are
// the same for every x, so the count is a sum over the shell's offsets of
// F(o) = #{x : col(x) = col(x + o)}.  F is computed once per distinct offset
// of all requested shells, then summed per shell.

static uint64_t pack_offset(const int o[4], const int dims[4], bool *zero) {
    uint64_t key = 0;
    *zero = true;
    for (int nu = 0; nu < 4; ++nu) {
        int c = o[nu] % dims[nu];
        if (c < 0) c += dims[nu];
        *zero = *zero && c == 0;
        key |= (uint64_t)c << (16 * nu);
    }
    return key;
}

static void shell_keys(const int dims[4], int mu, int p, int k, std::vector<uint64_t> &keys) {
    keys.clear();
    int rest[3], r = 0;
    for (int nu = 0; nu < 4; ++nu)
        if (nu != mu) rest[r++] = nu;
    for (int a = -k; a <= k; ++a)
        for (int b = -(k - abs(a)); b <= k - abs(a); ++b)
            for (int e = -(k - abs(a) - abs(b)); e <= k - abs(a) - abs(b); ++e) {
                const int t = k - abs(a) - abs(b) - abs(e);  // distance left along mu
                const int cand[4] = {p + t, p - t, t - p, -p - t};
                for (int q = 0; q < 4; ++q) {
                    const int om = cand[q];
                    if (std::min(abs(om - p), abs(om + p)) != t) continue;
                    int o[4];
                    o[mu] = om;
                    o[rest[0]] = a;
                    o[rest[1]] = b;
                    o[rest[2]] = e;
                    bool zero;
                    uint64_t key = pack_offset(o, dims, &zero);
                    if (!zero) keys.push_back(key);
                }
            }
    std::sort(keys.begin(), keys.end());
    keys.erase(std::unique(keys.begin(), keys.end()), keys.end());
}

#define PT_CLR_OB 8
#define PT_CLR_SITES 4096

// F(o) for a block of PT_CLR_OB offsets over a block of PT_CLR_SITES nodes:
// every thread keeps one counter per offset, warps reduce, the CTA adds one
// value per offset to F.
__global__ void __launch_bounds__(256) k_offset_matches(Geom g, const int32_t *__restrict__ col,
                                                        const uint2 *__restrict__ off, int n_off,
                                                        unsigned long long *__restrict__ F) {
    __shared__ uint2 so[PT_CLR_OB];
    __shared__ unsigned sc[PT_CLR_OB];
    const int o0 = blockIdx.y * PT_CLR_OB;
    const int nb = min(PT_CLR_OB, n_off - o0);
    if (threadIdx.x < PT_CLR_OB) {
        so[threadIdx.x] = (int)threadIdx.x < nb ? off[o0 + threadIdx.x] : make_uint2(0u, 0u);
        sc[threadIdx.x] = 0u;
    }
    __syncthreads();
    unsigned cnt[PT_CLR_OB];
#pragma unroll
    for (int o = 0; o < PT_CLR_OB; ++o) cnt[o] = 0u;
    const int begin = blockIdx.x * PT_CLR_SITES;
    const int end = min(g.N, begin + PT_CLR_SITES);
    for (int xs = begin + threadIdx.x; xs < end; xs += blockDim.x) {
        int x[4];
        site_coords(g, xs, x);
        const int cx = col[xs];
#pragma unroll
        for (int o = 0; o < PT_CLR_OB; ++o) cnt[o] += (unsigned)(col[walk_site(g, x, so[o])] == cx);
    }
#pragma unroll
    for (int o = 0; o < PT_CLR_OB; ++o) {
        unsigned v = __reduce_add_sync(0xffffffffu, cnt[o]);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&sc[o], v);
    }
    __syncthreads();
    if ((int)threadIdx.x < nb && sc[threadIdx.x]) atomicAdd(&F[o0 + threadIdx.x], (unsigned long long)sc[threadIdx.x]);
}

// one CTA per shell: the sum of F over the shell's offsets
__global__ void __launch_bounds__(256) k_shell_sums(const unsigned long long *__restrict__ F,
                                                    const int *__restrict__ idx, const int *__restrict__ start,
                                                    unsigned long long *__restrict__ out) {
    __shared__ unsigned long long sh[8];
    unsigned long long s = 0;
    for (int i = start[blockIdx.x] + threadIdx.x; i < start[blockIdx.x + 1]; i += blockDim.x) s += F[idx[i]];
    for (int d = 16; d; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        out[blockIdx.x] = t;
    }
}

extern "C" int pt_clearance(pt_ctx *c, const int dims[4], int mu, const int32_t *col_dev, const int *p_list, int n_p,
                            const int *k_list, int n_k, int64_t *matches_out, int64_t *shell_out) {
    PT_CHECK_ARG(c && dims && col_dev && p_list && k_list && matches_out && shell_out, "pt_clearance: NULL argument");
    PT_CHECK_ARG(mu >= 0 && mu <= 3 && n_p >= 1 && n_p <= 64 && n_k >= 1 && n_k <= 64,
                 "pt_clearance: mu in 0..3, 1 <= n_p, n_k <= 64");
    for (int nu = 0; nu < 4; ++nu)
        PT_CHECK_ARG(dims[nu] >= 1 && dims[nu] < 65536, "pt_clearance: lattice sides must be in 1..65535");
    for (int i = 0; i < n_p; ++i) PT_CHECK_ARG(p_list[i] >= 0 && p_list[i] <= 4096, "pt_clearance: bad p");
    for (int j = 0; j < n_k; ++j) PT_CHECK_ARG(k_list[j] >= 0 && k_list[j] <= 32, "pt_clearance: k in 0..32");
    PT_CUDA(cudaSetDevice(c->device));
    Geom g = make_geom(dims);
    const int n_pairs = n_p * n_k;
    std::vector<std::vector<uint64_t>> shells(n_pairs);
    std::vector<uint64_t> all;
    for (int i = 0; i < n_p; ++i)
        for (int j = 0; j < n_k; ++j) {
            shell_keys(dims, mu, p_list[i], k_list[j], shells[i * n_k + j]);
            all.insert(all.end(), shells[i * n_k + j].begin(), shells[i * n_k + j].end());
        }
    std::sort(all.begin(), all.end());
    all.erase(std::unique(all.begin(), all.end()), all.end());
    const int n_off = (int)all.size();
    PT_CHECK_ARG((n_off + PT_CLR_OB - 1) / PT_CLR_OB <= 65535, "pt_clearance: %d distinct offsets exceed one launch",
                 n_off);
    std::vector<int> start(n_pairs + 1, 0), idx;
    for (int q = 0; q < n_pairs; ++q) {
        for (uint64_t key : shells[q]) idx.push_back((int)(std::lower_bound(all.begin(), all.end(), key) - all.begin()));
        start[q + 1] = (int)idx.size();
        shell_out[q] = (int64_t)shells[q].size();
    }
    std::vector<uint2> off(n_off);
    for (int i = 0; i < n_off; ++i) off[i] = make_uint2((unsigned)all[i], (unsigned)(all[i] >> 32));
    auto al = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t off_b = al(off.size() * sizeof(uint2) + 8), F_b = al((size_t)n_off * 8 + 8),
                 idx_b = al(idx.size() * sizeof(int) + 4), st_b = al(start.size() * sizeof(int)),
                 out_b = al((size_t)n_pairs * 8);
    void *ws;
    int rc = pt_workspace(c, off_b + F_b + idx_b + st_b + out_b, &ws);
    if (rc) return rc;
    char *p = (char *)ws;
    uint2 *d_off = (uint2 *)p;
    unsigned long long *d_F = (unsigned long long *)(p + off_b);
    int *d_idx = (int *)(p + off_b + F_b);
    int *d_start = (int *)(p + off_b + F_b + idx_b);
    unsigned long long *d_out = (unsigned long long *)(p + off_b + F_b + idx_b + st_b);
    if (n_off) PT_CUDA(cudaMemcpyAsync(d_off, off.data(), off.size() * sizeof(uint2), cudaMemcpyHostToDevice, c->stream));
    if (!idx.empty())
        PT_CUDA(cudaMemcpyAsync(d_idx, idx.data(), idx.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    PT_CUDA(cudaMemcpyAsync(d_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice, c->stream));
    PT_CUDA(cudaMemsetAsync(d_F, 0, (size_t)n_off * 8 + 8, c->stream));
    if (n_off) {
        dim3 grid((unsigned)((g.N + PT_CLR_SITES - 1) / PT_CLR_SITES), (unsigned)((n_off + PT_CLR_OB - 1) / PT_CLR_OB));
        k_offset_matches<<<grid, 256, 0, c->stream>>>(g, col_dev, d_off, n_off, d_F);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
    }
    k_shell_sums<<<n_pairs, 256, 0, c->stream>>>(d_F, d_idx, d_start, d_out);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    std::vector<unsigned long long> h(n_pairs);
    PT_CUDA(cudaMemcpyAsync(h.data(), d_out, (size_t)n_pairs * 8, cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaStreamSynchronize(c->stream));
    for (int q = 0; q < n_pairs; ++q) matches_out[q] = (int64_t)h[q];
    return PT_OK;
}
