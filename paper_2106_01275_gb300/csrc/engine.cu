// Batched multi-RHS solver engine: every right-hand side (probe x set x
// dilution component, or a user column) is a task in a device queue; R
// "slots" hold the tasks in flight.  One engine iteration is a fixed sequence
// of kernels captured once into a CUDA graph and replayed:
//
//   schedule         retire finished slots, refill them from the queue, build work lists
//   contract         for converged slots: shifted-dot contraction v^H P_n x (Eqs. (1), (5))
//                    [trace mode], copy-out [solve mode]
//   outer_update     x64 += e  (FP64 defect-correction update)       / x64 = 0 at start
//   outer_residual   r64 = b - A x64 in FP64 (b regenerated from the counter-based
//                    noise, Eq. (5)), true relative residual, convergence -> contract,
//                    else restart the inner solve on r (rounded to the inner precision)
//   inner iteration  CG (Laplacian) or BiCGStab (Wilson) on A e = r in FP64, FP32 or
//                    BF16 storage, per-slot scalars in FP64
//
// Every kernel walks a device-built list of (slot, site block) work items
// with a grid sized to the GPU (persistent CTAs).  Per-slot reductions are
// deterministic: each item writes its partial sum, and the last item of a
// slot (atomic completion counter) sums the partials in a fixed order and
// advances the slot's state machine.  The host only replays the graph and
// reads one flag word per replay.
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "pt_common.cuh"

#define PT_BLOCK 256        // threads per engine work item

enum { PH_EMPTY = 0, PH_START = 1, PH_OUTER = 2, PH_INNER = 3, PH_CONTRACT = 4, PH_DONE = 5 };
enum { MODE_TRACE = 0, MODE_SOLVE = 1, MODE_GRAD = 2 };
enum { LIST_CONTRACT = 0, LIST_OUTER = 1, LIST_INNER = 2 };
enum { TASK_ADJ = 1 };      // source is P^T v (with g5 for Wilson)

struct Slot {
    int task, phase, inner_it, total_it;
    int outer_it, pad0, pad1, pad2;
    double bnorm2, rr, rr0, target2;
    double relres, pad3;
    Cx<double> alpha, beta, omega, rho;
};

struct Task {
    int set, colour, comp, flags;
    int cidx, pad0, pad1, pad2;   // cidx: which colouring (multi-colouring runs)
};

struct TaskStat {
    int iters, outer;
    double relres;
};

struct EP {
    Geom g;
    int kind, nsb, R, gs, vec4;
    int bs, spt;               // threads of an item kernel's CTA; sites per thread (an item is bs x spt sites)
    int eo;                    // Laplacian on the even Schur complement (inner vectors on the even sites)
    int nsite;                 // entries of a slot field: N, or N / 2 in even-odd mode
    int rhs_block;             // Wilson applies: right-hand sides per item (1 or 2)
    int overlap;               // groups run as graph branches: the inner list holds PH_INNER slots only
    // nested trace mode (n_lev > 0): the tasks are the classes of the finest of
    // n_lev nested colourings lev_cols [n_lev][N]; output q = l * n_pr + n is the
    // contraction with the level-l probe (ancestor class lev_anc[l][colour])
    int n_lev, n_pr, m_fin;
    const int32_t *lev_cols;
    const int *lev_anc;
    int64_t L;                 // reals per slot field
    double diag, kappa;
    int antip;
    const void *U;             // links in the inner precision
    const double *U64;         // links in FP64
    int clover;                // even-odd Wilson with a clover term: the packed chiral blocks below
    const float4 *CL32;        // 1 + C (even), (1 + C)^{-1} (odd) for FP32 / BF16 inner storage
    const double2 *CL64;       // the same in FP64 (and 1 + C on the odd sites)
    int mode;
    const int32_t *col;
    uint64_t seed;
    int noise, mu, n_p, dilute, pshift;
    int p[PT_MAX_P];
    const Task *tasks;
    int n_tasks;
    const double *B_user;      // solve mode: user layout sources
    double *X_user;            // solve mode: user layout solutions
    double *x64;
    double *t64;               // even-odd: H_oe x64 (Laplacian) / D_oe x64 (Wilson) on the odd sites (FP64)
    double *b64;               // even-odd: b'_e of the slot's task (FP64; b_e + H_eo b_o / d, resp. + kappa D_eo b_o)
    void *e, *r, *pv, *q, *s, *t, *r0, *p1;   // p1: second CG direction buffer; even-odd: t = H_oe p (odd sites)
    Slot *slots;
    double *partials;
    int *counters, *lists, *counts, *head, *flags;
    TaskStat *tstat;
    double *task_out;          // trace mode: [n_tasks][n_p] complex
    double tol, delta;
    int maxit, max_inner;
};

#define FLAG_DONE 0
#define FLAG_NUMERIC 1
#define FLAG_NOCONV 2

// ------------------------------------------------------------------ field access
template <int KIND, typename S>
struct Fld {
    static constexpr int NC = KIND ? 12 : 1;
    typedef typename ArithT<S>::T R;
    __device__ __forceinline__ static Cx<R> ld(const S *f, int N, int c, int idx) {
        if constexpr (KIND == 0) return Cx<R>{(R)ld_real(f, (size_t)idx), R(0)};
        else return ld_cx<S, R>(f, N, c, idx);
    }
    __device__ __forceinline__ static void st(S *f, int N, int c, int idx, Cx<R> v) {
        if constexpr (KIND == 0) st_real(f, (size_t)idx, v.re);
        else st_cx<S, R>(f, N, c, idx, v);
    }
};

template <typename T>
__device__ __forceinline__ T *slot_ptr(void *base, int j, int64_t L) {
    return reinterpret_cast<T *>(base) + (size_t)j * L;
}
template <typename T>
__device__ __forceinline__ const T *slot_cptr(const void *base, int j, int64_t L) {
    return reinterpret_cast<const T *>(base) + (size_t)j * L;
}

// y = A f at one site (all NC components) in arithmetic R
template <int KIND, typename R, typename S, typename LS>
__device__ __forceinline__ void apply_site(const EP &P, const S *f, const LS *U, int idx, const int x[4],
                                           Cx<R> out[Fld<KIND, S>::NC]) {
    if constexpr (KIND == 0) {
        out[0] = Cx<R>{lap_site<R, S>(P.g, f, (R)P.diag, idx, x), R(0)};
    } else {
        Cx<R> acc[4][3];
        wilson_hop_site<R, S, LS>(P.g, f, U, P.antip, idx, x, acc);
        Cx<R> ps[4][3];
        load_spinor<S, R>(f, P.g.N, idx, ps);
        const R kap = (R)P.kappa;
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) out[3 * s + a] = csub(ps[s][a], cscale(acc[s][a], kap));
    }
}

// source b(x, a) of a task
template <int KIND>
__device__ __forceinline__ Cx<double> source_val(const EP &P, const Task &tk, uint64_t key, int idx,
                                                 const int x[4], int a) {
    const int dof = KIND ? 12 : 1;
    if (P.mode == MODE_SOLVE) {
        const double *b = P.B_user + ((size_t)tk.set * P.g.N + idx) * dof * (KIND ? 2 : 1);
        if constexpr (KIND == 0) return Cx<double>{b[0], 0.0};
        else return Cx<double>{b[2 * a], b[2 * a + 1]};
    }
    int src = idx;
    double sg = 1.0;
    if (tk.flags & TASK_ADJ) {
        src = shift_site(P.g, idx, x, P.mu, -P.pshift);      // (P^T v)(x) = v(x - p)
        if (KIND && a >= 6) sg = -1.0;                       // g5 = diag(1, 1, -1, -1)
    }
    if (P.col[(size_t)tk.cidx * P.g.N + src] != tk.colour) return Cx<double>{0.0, 0.0};
    Cx<double> z;
    if (P.dilute) {
        if (a != tk.comp) return Cx<double>{0.0, 0.0};
        z = pt_noise(key, (uint64_t)src, P.noise);
    } else {
        z = pt_noise(key, (uint64_t)src * dof + a, P.noise);
    }
    return Cx<double>{sg * z.re, sg * z.im};
}

// site index and coordinate along mu of x + p e_mu for 0 <= p < D_mu (the
// engine reduces its displacements once on the host): an add and a
// conditional subtract instead of a modulo
__device__ __forceinline__ int shift_fwd(const Geom &g, int idx, const int x[4], int mu, int p, int *c_out) {
    int c = x[mu] + p;
    if (c >= g.D[mu]) c -= g.D[mu];
    *c_out = c;
    return idx + (c - x[mu]) * g.stride[mu];
}

// ------------------------------------------------------------------ work items and reductions
// An item is one slot's block of bs x spt consecutive sites, processed by one
// CTA of bs threads (spt sites per thread; by default PT_BLOCK threads and
// Tile<KIND>::SPT sites, the autotuner may choose others).  A reduction stores one
// partial sum per item (plain stores: the kernel boundary orders them); a
// finalize kernel with one warp per slot adds the slot's nsb partials in a
// fixed order (deterministic) and advances the slot's state machine.
template <int KIND>
struct Tile {
    static constexpr int SPT = KIND ? 1 : 8;
    static constexpr int SITES = PT_BLOCK * SPT;
};

// Item order: slots are taken in groups of P.gs; inside a group the items run
// site-block-major, so that consecutive CTAs share a site block (the links of
// the Wilson operator are reused across the group from L2) while a slot's halo
// blocks are visited close in time (gs = 1: slot-major, for the Laplacian).
#define ITEM_LOOP(LIST)                                                         \
    const int cnt = P.counts[LIST];                                             \
    const int *lst = P.lists + (size_t)(LIST) * P.R;                            \
    const int64_t n_items = (int64_t)cnt * P.nsb;                               \
    const int64_t gitems_ = (int64_t)P.gs * P.nsb;                              \
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {              \
        const int64_t g_ = it / gitems_;                                        \
        const int base_ = (int)(g_ * P.gs);                                     \
        const int gsz_ = min(P.gs, cnt - base_);                                \
        const int rem_ = (int)(it - g_ * gitems_);                              \
        const int b = rem_ / gsz_;                                              \
        const int j = lst[base_ + rem_ % gsz_];
#define ITEM_LOOP_END }

#define SITE_LOOP(KIND)                                                         \
    for (int k_ = 0; k_ < ((KIND) ? 1 : P.spt); ++k_) {                         \
        const int idx = b * (((KIND) ? 1 : P.spt) * P.bs) + k_ * P.bs + (int)threadIdx.x; \
        if (idx >= N) continue;
#define SITE_LOOP_END }

template <int K>
__device__ __forceinline__ void item_store(const EP &P, int j, int b, double v[K], double *sh) {
    block_sum<K>(v, sh);
    if (threadIdx.x == 0) {
        double *dst = P.partials + ((size_t)j * P.nsb + b) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) dst[k] = v[k];
    }
}

// per-thread partials accumulated in the arithmetic type R (FP32 for the
// FP32 / BF16 inner solves: the FP64 pipe of GB300 is too narrow for a
// per-site FP64 sum), widened to FP64 for the block and slot reductions
template <int K, typename R>
__device__ __forceinline__ void item_store_r(const EP &P, int j, int b, R vr[K], double *sh) {
    if constexpr (std::is_same<R, double>::value) {
        item_store<K>(P, j, b, vr, sh);
    } else {
        // warp tree in R, then the (at most 32) warp sums added in FP64 in a fixed order
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
        for (int k = 0; k < K; ++k)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) vr[k] += __shfl_down_sync(0xffffffffu, vr[k], o);
        __syncthreads();
        if (lane == 0)
#pragma unroll
            for (int k = 0; k < K; ++k) sh[warp * K + k] = (double)vr[k];
        __syncthreads();
        if (threadIdx.x == 0) {
            double *dst = P.partials + ((size_t)j * P.nsb + b) * K;
#pragma unroll
            for (int k = 0; k < K; ++k) {
                double s = 0.0;
                for (int w = 0; w < nw; ++w) s += sh[w * K + k];
                dst[k] = s;
            }
        }
    }
}

// contraction partials: only the first K = 2 n_p of the 2 PT_MAX_P entries are
// reduced (FP64 throughout: these are the trace accumulations); the rest are zero
template <int MAXQ>
__device__ __forceinline__ void item_store_contract(const EP &P, int j, int b, double acc[2 * MAXQ], int K,
                                                    double *sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < 2 * MAXQ; ++k) {
        if (k < K) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[k] += __shfl_down_sync(0xffffffffu, acc[k], o);
        }
    }
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < 2 * MAXQ; ++k)
            if (k < K) sh[warp * 2 * PT_MAX_P + k] = acc[k];
    __syncthreads();
    if (threadIdx.x == 0) {
        double *dst = P.partials + ((size_t)j * P.nsb + b) * 2 * PT_MAX_P;
        for (int k = 0; k < 2 * PT_MAX_P; ++k) {
            double s = 0.0;
            if (k < K)
                for (int w = 0; w < nw; ++w) s += sh[w * 2 * PT_MAX_P + k];
            dst[k] = s;
        }
    }
}

#define WARP_LOOP(LIST)                                                         \
    const int cnt = P.counts[LIST];                                             \
    const int *lst = P.lists + (size_t)(LIST) * P.R;                            \
    const int lane = threadIdx.x & 31;                                          \
    const int wstride = (int)((gridDim.x * blockDim.x) >> 5);                   \
    for (int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); w < cnt; w += wstride) { \
        const int j = lst[w];                                                   \
        Slot &st = P.slots[j];
#define WARP_LOOP_END }

// all lanes receive the slot's total (fixed summation order)
template <int K>
__device__ __forceinline__ void warp_total(const EP &P, int j, double tot[K]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int k = 0; k < K; ++k) tot[k] = 0.0;
    const double *src = P.partials + (size_t)j * P.nsb * K;
    for (int i = lane; i < P.nsb; i += 32)
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] += src[(size_t)i * K + k];
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) tot[k] += __shfl_xor_sync(0xffffffffu, tot[k], o);
}

// value rounded to the storage type S (and back to the arithmetic type)
template <typename S, typename R>
__device__ __forceinline__ R rnd(R v) {
    if constexpr (std::is_same<S, __nv_bfloat16>::value) return __bfloat162float(__float2bfloat16_rn(v));
    else return v;
}

// ------------------------------------------------------------------ schedule
__device__ int block_exclusive_scan(int v, int *sh, int &total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    __syncthreads();
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int w = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;
    }
    __syncthreads();
    int prefix = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    total = sh[nw - 1];
    __syncthreads();
    return prefix;
}

__global__ void __launch_bounds__(1024) k_schedule(EP P) {
    __shared__ int sh[32];
    __shared__ int s_head, s_cnt[3], s_busy;
    if (threadIdx.x == 0) { s_head = *P.head; s_cnt[0] = s_cnt[1] = s_cnt[2] = 0; s_busy = 0; }
    __syncthreads();
    for (int base = 0; base < P.R; base += blockDim.x) {
        int j = base + threadIdx.x;
        int ph = (j < P.R) ? P.slots[j].phase : -1;
        int need = (ph == PH_EMPTY || ph == PH_DONE) && (P.mode != MODE_GRAD || ph == PH_EMPTY);
        int total;
        int rank = block_exclusive_scan(need, sh, total);
        if (need) {
            int t = s_head + rank;
            Slot &st = P.slots[j];
            if (t < P.n_tasks) {
                st.task = t; st.phase = PH_START; st.inner_it = 0; st.total_it = 0; st.outer_it = 0;
                ph = PH_START;
            } else {
                if (ph == PH_DONE && P.mode != MODE_GRAD) { st.phase = PH_EMPTY; st.task = -1; }
                ph = (ph == PH_DONE) ? PH_DONE : PH_EMPTY;
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) s_head = min(s_head + total, P.n_tasks);
        __syncthreads();
        // work lists
        int in_c = (ph == PH_CONTRACT);
        int in_o = (ph == PH_START || ph == PH_OUTER);
        // serial iterations let a slot leaving the outer step start its inner solve at once; with
        // the groups as concurrent branches the inner list must not share slots with the outer one
        int in_i = P.overlap ? (ph == PH_INNER) : (ph == PH_START || ph == PH_OUTER || ph == PH_INNER);
        int busy = (ph >= PH_START && ph <= PH_CONTRACT);
        int tc, to, ti, tb;
        int rc = block_exclusive_scan(in_c, sh, tc);
        int ro = block_exclusive_scan(in_o, sh, to);
        int ri = block_exclusive_scan(in_i, sh, ti);
        block_exclusive_scan(busy, sh, tb);
        if (in_c) P.lists[LIST_CONTRACT * P.R + s_cnt[0] + rc] = j;
        if (in_o) P.lists[LIST_OUTER * P.R + s_cnt[1] + ro] = j;
        if (in_i) P.lists[LIST_INNER * P.R + s_cnt[2] + ri] = j;
        __syncthreads();
        if (threadIdx.x == 0) { s_cnt[0] += tc; s_cnt[1] += to; s_cnt[2] += ti; s_busy += tb; }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        *P.head = s_head;
        P.counts[0] = s_cnt[0]; P.counts[1] = s_cnt[1]; P.counts[2] = s_cnt[2];
        P.flags[FLAG_DONE] = (s_head >= P.n_tasks && s_busy == 0) ? 1 : 0;
    }
}

// ------------------------------------------------------------------ contract / copy-out
// trace mode: q_n = sum_x conj(v(x)) x(x + p_n e_mu) for every displacement
// (the shifted dot of Eq. (1) with P_{p_n}); solve mode: copy x to the user.
// MAXQ: compiled bound on the outputs per solve (displacements x nested levels)
template <int KIND, int MAXQ>
__global__ void __launch_bounds__(PT_BLOCK) k_contract(EP P) {
    __shared__ double sh[32 * 2 * PT_MAX_P];
    const int N = P.g.N;
    ITEM_LOOP(LIST_CONTRACT)
        const Slot &st = P.slots[j];
        if (st.phase != PH_CONTRACT) continue;
        const Task tk = P.tasks[st.task];
        const double *x = P.x64 + (size_t)j * P.L;
        if (P.mode == MODE_SOLVE) {
            SITE_LOOP(KIND)
                if constexpr (KIND == 0) {
                    P.X_user[(size_t)tk.set * N + idx] = x[idx];
                } else {
                    double *dst = P.X_user + ((size_t)tk.set * N + idx) * 24;
                    for (int c = 0; c < 12; ++c) {
                        Cx<double> v = ld_cx<double, double>(x, N, c, idx);
                        dst[2 * c] = v.re;
                        dst[2 * c + 1] = v.im;
                    }
                }
            SITE_LOOP_END
            continue;
        }
        double acc[2 * MAXQ];
#pragma unroll
        for (int n = 0; n < 2 * MAXQ; ++n) acc[n] = 0.0;
        const uint64_t key = pt_set_key(P.seed, tk.set);
        const int32_t *col = P.col + (size_t)tk.cidx * N;
        SITE_LOOP(KIND)
            if (P.n_lev) {                 // the coarsest ancestor class holds every finer one
                if (P.lev_cols[idx] != P.lev_anc[tk.colour]) continue;
            } else if (col[idx] != tk.colour) {
                continue;
            }
            int xc[4];
            site_coords(P.g, idx, xc);
            const int dof = KIND ? 12 : 1;
            for (int a = 0; a < dof; ++a) {
                if (P.dilute && a != tk.comp) continue;
                Cx<double> z = P.dilute ? pt_noise(key, (uint64_t)idx, P.noise)
                                        : pt_noise(key, (uint64_t)idx * dof + a, P.noise);
#pragma unroll
                for (int n = 0; n < MAXQ; ++n) {
                    if (n >= P.n_p) break;
                    if (P.n_lev) {
                        const int l = n / P.n_pr;
                        if (l > 0 && P.lev_cols[(size_t)l * N + idx] != P.lev_anc[(size_t)l * P.m_fin + tk.colour])
                            continue;
                    }
                    int cm;
                    const int y = shift_fwd(P.g, idx, xc, P.mu, P.p[n], &cm);
                    Cx<double> q = cconjmul(z, Fld<KIND, double>::ld(x, N, a, y));
                    acc[2 * n] += q.re;
                    acc[2 * n + 1] += q.im;
                }
            }
        SITE_LOOP_END
        item_store_contract<MAXQ>(P, j, b, acc, 2 * P.n_p, sh);
    ITEM_LOOP_END
}

__global__ void k_fin_contract(EP P) {
    WARP_LOOP(LIST_CONTRACT)
        if (st.phase != PH_CONTRACT) continue;
        if (P.mode == MODE_TRACE) {
            double tot[2 * PT_MAX_P];
            warp_total<2 * PT_MAX_P>(P, j, tot);
            if (lane == 0)
                for (int n = 0; n < P.n_p; ++n) {
                    P.task_out[((size_t)st.task * P.n_p + n) * 2] = tot[2 * n];
                    P.task_out[((size_t)st.task * P.n_p + n) * 2 + 1] = tot[2 * n + 1];
                }
        }
        __syncwarp();
        if (lane == 0) st.phase = PH_DONE;
    WARP_LOOP_END
}

// ------------------------------------------------------------------ outer (FP64) steps
// x64 += e (FP64 defect-correction update); x64 = 0 for a newly started task
template <int KIND, typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_outer_update(EP P) {
    typedef Fld<KIND, S> F;
    const int N = P.nsite;            // field entries per slot (N/2 in even-odd mode)
    ITEM_LOOP(LIST_OUTER)
        const int ph = P.slots[j].phase;
        if (ph != PH_START && ph != PH_OUTER) continue;
        double *x = P.x64 + (size_t)j * P.L;
        const S *e = slot_cptr<S>(P.e, j, P.L);
        SITE_LOOP(KIND)
            for (int c = 0; c < F::NC; ++c) {
                Cx<double> v = {0.0, 0.0};
                if (ph == PH_OUTER) {
                    Cx<double> xv = Fld<KIND, double>::ld(x, N, c, idx);
                    auto ev = F::ld(e, N, c, idx);
                    v = Cx<double>{xv.re + (double)ev.re, xv.im + (double)ev.im};
                }
                Fld<KIND, double>::st(x, N, c, idx, v);
            }
        SITE_LOOP_END
    ITEM_LOOP_END
}

// r64 = b - A x64 in FP64; r = (S) r64 starts the inner solve (e = 0);
// partials: |r64|^2, |b|^2, |r|^2 (of the rounded r)
template <int KIND, typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_outer_residual(EP P) {
    typedef Fld<KIND, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 3];
    const int N = P.g.N;
    ITEM_LOOP(LIST_OUTER)
        const Slot &st = P.slots[j];
        const int ph = st.phase;
        if (ph != PH_START && ph != PH_OUTER) continue;
        const Task tk = P.tasks[st.task];
        const uint64_t key = (P.mode == MODE_SOLVE) ? 0 : pt_set_key(P.seed, tk.set);
        S *r = slot_ptr<S>(P.r, j, P.L);
        S *pv = slot_ptr<S>(P.pv, j, P.L);
        S *e = slot_ptr<S>(P.e, j, P.L);
        S *r0 = KIND ? slot_ptr<S>(P.r0, j, P.L) : nullptr;
        double v[3] = {0.0, 0.0, 0.0};
        SITE_LOOP(KIND)
            int xc[4];
            site_coords(P.g, idx, xc);
            Cx<double> ax[F::NC];
            if (ph == PH_OUTER) {
                apply_site<KIND, double, double, double>(P, P.x64 + (size_t)j * P.L, P.U64, idx, xc, ax);
            } else {
#pragma unroll
                for (int c = 0; c < F::NC; ++c) ax[c] = Cx<double>{0.0, 0.0};
            }
            for (int c = 0; c < F::NC; ++c) {
                Cx<double> bv = source_val<KIND>(P, tk, key, idx, xc, c);
                Cx<double> rv = csub(bv, ax[c]);
                v[0] += rv.re * rv.re + rv.im * rv.im;
                v[1] += bv.re * bv.re + bv.im * bv.im;
                Cx<R> rs = Cx<R>{rnd<S, R>((R)rv.re), rnd<S, R>((R)rv.im)};
                F::st(r, N, c, idx, rs);
                if constexpr (KIND == 1) {
                    F::st(pv, N, c, idx, rs);
                    F::st(r0, N, c, idx, rs);
                }
                F::st(e, N, c, idx, Cx<R>{R(0), R(0)});
                v[2] += (double)rs.re * (double)rs.re + (double)rs.im * (double)rs.im;
            }
        SITE_LOOP_END
        item_store<3>(P, j, b, v, sh);
    ITEM_LOOP_END
}

__global__ void k_fin_outer(EP P) {
    WARP_LOOP(LIST_OUTER)
        const int ph = st.phase;
        if (ph != PH_START && ph != PH_OUTER) continue;
        double tot[3];
        warp_total<3>(P, j, tot);
        if (lane == 0) {
            if (ph == PH_START) st.bnorm2 = tot[1];
            const double b2 = st.bnorm2;
            const double rel = b2 > 0.0 ? sqrt(tot[0] / b2) : 0.0;
            st.relres = rel;
            st.outer_it += 1;
            const bool finite = isfinite(tot[0]);
            if (!finite) atomicOr(&P.flags[FLAG_NUMERIC], 1);
            const bool conv = (b2 == 0.0) || rel <= P.tol;
            if (conv || !finite || st.total_it >= P.maxit) {
                if (!conv && finite) atomicAdd(&P.flags[FLAG_NOCONV], 1);
                P.tstat[st.task] = TaskStat{st.total_it, st.outer_it, rel};
                st.phase = (P.mode == MODE_GRAD) ? PH_DONE : PH_CONTRACT;
            } else {
                st.phase = PH_INNER;
                st.inner_it = 0;
                st.rr = tot[2];
                st.rr0 = tot[2];
                st.rho = Cx<double>{tot[2], 0.0};
                st.beta = Cx<double>{0.0, 0.0};
                st.target2 = fmax(P.delta * P.delta * tot[2], 0.25 * P.tol * P.tol * b2);
            }
        }
    WARP_LOOP_END
}

// ------------------------------------------------------------------ CG (Laplacian)
// Fused direction update and stencil: with i = inner iteration,
//   p_i = r + beta p_{i-1}  (p_0 = r)   -- recomputed at the neighbours, stored at x
//   q   = A p_i,  partial p_i . q
// p alternates between two buffers (pv, p1) so that no CTA reads a value
// another CTA is overwriting.
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_cg_apply(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32];
    const int N = P.g.N;
    const R diag = (R)P.diag;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int i = st.inner_it;
        const R be = (R)st.beta.re;
        const bool first = (i == 0);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *pold = slot_cptr<S>((i & 1) ? P.p1 : P.pv, j, P.L);
        S *pnew = slot_ptr<S>((i & 1) ? P.pv : P.p1, j, P.L);
        S *q = slot_ptr<S>(P.q, j, P.L);
        R vr[1] = {R(0)};
        SITE_LOOP(0)
            int xc[4];
            site_coords(P.g, idx, xc);
            auto pn = [&](int y) -> R {
                R rv = ld_real(r, (size_t)y);
                return first ? rv : rnd<S, R>(rv + be * (R)ld_real(pold, (size_t)y));
            };
            const R pc = pn(idx);
            R nb = R(0);
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                nb += pn(nb_fwd(P.g, idx, xc, mu));
                nb += pn(nb_bwd(P.g, idx, xc, mu));
            }
            const R qv = rnd<S, R>(diag * pc - nb);
            st_real(pnew, (size_t)idx, pc);
            st_real(q, (size_t)idx, qv);
            vr[0] += pc * qv;
        SITE_LOOP_END
        item_store_r<1>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

__global__ void k_fin_cg_alpha(EP P) {
    WARP_LOOP(LIST_INNER)
        if (st.phase != PH_INNER) continue;
        double tot[1];
        warp_total<1>(P, j, tot);
        if (lane == 0) {
            if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
                atomicOr(&P.flags[FLAG_NUMERIC], 2);
                st.phase = PH_OUTER;                     // restart from the true residual
            } else {
                st.alpha = Cx<double>{st.rr / tot[0], 0.0};
            }
        }
    WARP_LOOP_END
}

// e += alpha p_i;  r -= alpha q;  partial |r|^2
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_cg_update(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32];
    const int N = P.nsite;            // field entries per slot (N/2 in even-odd mode)
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const R al = (R)st.alpha.re;
        S *e = slot_ptr<S>(P.e, j, P.L);
        S *r = slot_ptr<S>(P.r, j, P.L);
        const S *pc = slot_cptr<S>((st.inner_it & 1) ? P.pv : P.p1, j, P.L);
        const S *q = slot_cptr<S>(P.q, j, P.L);
        R vr[1] = {R(0)};
        SITE_LOOP(0)
            const R ev = rnd<S, R>((R)ld_real(e, (size_t)idx) + al * (R)ld_real(pc, (size_t)idx));
            const R rv = rnd<S, R>((R)ld_real(r, (size_t)idx) - al * (R)ld_real(q, (size_t)idx));
            st_real(e, (size_t)idx, ev);
            st_real(r, (size_t)idx, rv);
            vr[0] += rv * rv;
        SITE_LOOP_END
        item_store_r<1>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

__global__ void k_fin_cg_beta(EP P) {
    WARP_LOOP(LIST_INNER)
        if (st.phase != PH_INNER) continue;
        double tot[1];
        warp_total<1>(P, j, tot);
        if (lane == 0) {
            st.inner_it += 1;
            st.total_it += 1;
            if (tot[0] <= st.target2 || st.inner_it >= P.max_inner || st.total_it >= P.maxit || !isfinite(tot[0])) {
                st.phase = PH_OUTER;
            } else {
                st.beta = Cx<double>{tot[0] / st.rr, 0.0};
                st.rr = tot[0];
            }
        }
    WARP_LOOP_END
}

// ------------------------------------------------------------------ CG, four sites per thread
// Fast path when D_0 is a multiple of 4: a thread owns the quad of sites
// 4m .. 4m+3 of one x row.  The quad and its y, z, t neighbour quads are
// vector loads (16 B for FP32, 8 B for BF16, 2 x 16 B for FP64); the two x
// neighbours outside the quad are scalar loads.  Same arithmetic as the
// one-site kernels above, so the two paths give identical results.
template <typename S> struct Quad;
template <> struct Quad<float> {
    __device__ __forceinline__ static void ld(const float *p, int i, float v[4]) {
        const float4 a = *reinterpret_cast<const float4 *>(p + i);
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    }
    __device__ __forceinline__ static void st(float *p, int i, const float v[4]) {
        *reinterpret_cast<float4 *>(p + i) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Quad<double> {
    __device__ __forceinline__ static void ld(const double *p, int i, double v[4]) {
        const double2 a = *reinterpret_cast<const double2 *>(p + i);
        const double2 c = *reinterpret_cast<const double2 *>(p + i + 2);
        v[0] = a.x; v[1] = a.y; v[2] = c.x; v[3] = c.y;
    }
    __device__ __forceinline__ static void st(double *p, int i, const double v[4]) {
        *reinterpret_cast<double2 *>(p + i) = make_double2(v[0], v[1]);
        *reinterpret_cast<double2 *>(p + i + 2) = make_double2(v[2], v[3]);
    }
};
template <> struct Quad<__nv_bfloat16> {
    __device__ __forceinline__ static void ld(const __nv_bfloat16 *p, int i, float v[4]) {
        const uint2 a = *reinterpret_cast<const uint2 *>(p + i);
        const float2 lo = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&a.x));
        const float2 hi = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162 *>(&a.y));
        v[0] = lo.x; v[1] = lo.y; v[2] = hi.x; v[3] = hi.y;
    }
    __device__ __forceinline__ static void st(__nv_bfloat16 *p, int i, const float v[4]) {
        __nv_bfloat162 lo = __floats2bfloat162_rn(v[0], v[1]);
        __nv_bfloat162 hi = __floats2bfloat162_rn(v[2], v[3]);
        uint2 a;
        a.x = *reinterpret_cast<uint32_t *>(&lo);
        a.y = *reinterpret_cast<uint32_t *>(&hi);
        *reinterpret_cast<uint2 *>(p + i) = a;
    }
};

#define QUAD_LOOP                                                               \
    for (int k_ = 0; k_ < P.spt / 4; ++k_) {                                    \
        const int idx = 4 * (b * (P.spt / 4 * P.bs) + k_ * P.bs + (int)threadIdx.x); \
        if (idx >= N) continue;
#define QUAD_LOOP_END }

template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_cg_apply_v4(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32];
    const int N = P.g.N;
    const int D0 = P.g.D[0];
    const R diag = (R)P.diag;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int i = st.inner_it;
        const R be = (R)st.beta.re;
        const bool first = (i == 0);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *pold = slot_cptr<S>((i & 1) ? P.p1 : P.pv, j, P.L);
        S *pnew = slot_ptr<S>((i & 1) ? P.pv : P.p1, j, P.L);
        S *q = slot_ptr<S>(P.q, j, P.L);
        R vr[1] = {R(0)};
        QUAD_LOOP
            int xc[4];
            site_coords(P.g, idx, xc);
            auto pquad = [&](int y, R out[4]) {
                Quad<S>::ld(r, y, out);
                if (!first) {
                    R pp[4];
                    Quad<S>::ld(pold, y, pp);
#pragma unroll
                    for (int c = 0; c < 4; ++c) out[c] = rnd<S, R>(out[c] + be * pp[c]);
                }
            };
            auto pone = [&](int y) -> R {
                R rv = ld_real(r, (size_t)y);
                return first ? rv : rnd<S, R>(rv + be * (R)ld_real(pold, (size_t)y));
            };
            R pc[4], t[4];
            pquad(idx, pc);
            const R left = pone(xc[0] == 0 ? idx + D0 - 1 : idx - 1);
            const R right = pone(xc[0] + 4 == D0 ? idx + 4 - D0 : idx + 4);
            // neighbours summed in the order of the one-site kernel: x+, x-, y+, y-, z+, z-, t+, t-
            R acc[4] = {pc[1] + left, pc[2] + pc[0], pc[3] + pc[1], right + pc[2]};
#pragma unroll
            for (int mu = 1; mu < 4; ++mu) {
                pquad(nb_fwd(P.g, idx, xc, mu), t);
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] += t[c];
                pquad(nb_bwd(P.g, idx, xc, mu), t);
#pragma unroll
                for (int c = 0; c < 4; ++c) acc[c] += t[c];
            }
            R qv[4];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                qv[c] = rnd<S, R>(diag * pc[c] - acc[c]);
                vr[0] += pc[c] * qv[c];
            }
            Quad<S>::st(pnew, idx, pc);
            Quad<S>::st(q, idx, qv);
        QUAD_LOOP_END
        item_store_r<1>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_cg_update_v4(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32];
    const int N = P.nsite;            // field entries per slot (N/2 in even-odd mode)
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const R al = (R)st.alpha.re;
        S *e = slot_ptr<S>(P.e, j, P.L);
        S *r = slot_ptr<S>(P.r, j, P.L);
        const S *pc = slot_cptr<S>((st.inner_it & 1) ? P.pv : P.p1, j, P.L);
        const S *q = slot_cptr<S>(P.q, j, P.L);
        R vr[1] = {R(0)};
        QUAD_LOOP
            R ev[4], pv[4], qv[4], rv[4];
            Quad<S>::ld(e, idx, ev);
            Quad<S>::ld(pc, idx, pv);
            Quad<S>::ld(q, idx, qv);
            Quad<S>::ld(r, idx, rv);
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                ev[c] = rnd<S, R>(ev[c] + al * pv[c]);
                rv[c] = rnd<S, R>(rv[c] - al * qv[c]);
                vr[0] += rv[c] * rv[c];
            }
            Quad<S>::st(e, idx, ev);
            Quad<S>::st(r, idx, rv);
        QUAD_LOOP_END
        item_store_r<1>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

// ------------------------------------------------------------------ even-odd CG (Laplacian)
// With every lattice side even the Laplacian splits by site parity,
// A = [[d, -H_eo], [-H_oe, d]] with d = 8 + m^2 and H the sum of the eight
// hops, and A x = b is solved through the Schur complement on the even sites:
//   S x_e = b'_e,  S = d - H_eo H_oe / d,  b'_e = b_e + H_eo b_o / d,
//   x_o = (b_o + H_oe x_e) / d.
// S is about four times better conditioned than A, so CG needs about half
// the iterations.  The inner vectors e, r, p, q live on the even sites and
// t = H_oe p on the odd ones.  A half field holds the sites of one parity in
// storage order: with D_0 even, site i is entry i >> 1 of its parity's field.
// One inner iteration is three kernels:
//   k_eo_hop     odd entries:  t = H_oe p_i, with p_i = r + beta p_{i-1} formed
//                at the eight even neighbours (as in k_cg_apply)
//   k_eo_apply   even entries: p_i stored, q = S p_i = d p_i - H_eo t / d,
//                partial p_i . q
//   k_cg_update  even entries: e += alpha p_i, r -= alpha q, partial |r|^2
// which moves 6 + 10 + 12 = 28 bytes per lattice site in FP32 (40 on the full
// system).  The FP64 outer step forms t64 = H_oe x64 on the odd entries, then
// r = b'_e - S x64 on the even ones, with b'_e formed from the regenerated
// noise when the task starts and kept in FP64; its
// |b|^2 is that of the whole source (both parities), so the stopping test is
// the full system's ||b - A x|| / ||b|| (r_o = 0 once x_o is rebuilt).  The
// contraction reads x_o = (b_o + t64) / d wherever it reads an odd site
// (t64 = H_oe x64 of the final x64: a slot converges right after the outer
// step that formed it).

// storage index and coordinates of entry h of the half field of parity par
__device__ __forceinline__ int half_site(const Geom &g, int par, int h, int x[4]) {
    const int q0 = fdiv(g.fd[0], 2 * h);            // row of sites 2h and 2h + 1 (D_0 even)
    const int x0e = 2 * h - q0 * g.D[0];
    const int q1 = fdiv(g.fd[1], q0);
    x[1] = q0 - q1 * g.D[1];
    const int q2 = fdiv(g.fd[2], q1);
    x[2] = q1 - q2 * g.D[2];
    x[3] = q2;
    const int b = (par ^ (x[1] + x[2] + x[3])) & 1;  // x_0 parity that gives the site parity par
    x[0] = x0e + b;
    return 2 * h + b;
}

// sum over the eight neighbours of site i (coordinates x) of f, a half field
// of the other parity
template <typename S, typename R>
__device__ __forceinline__ R half_nbsum(const Geom &g, const S *f, int i, const int x[4]) {
    R s = R(0);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        s += (R)ld_real(f, (size_t)(nb_fwd(g, i, x, mu) >> 1));
        s += (R)ld_real(f, (size_t)(nb_bwd(g, i, x, mu) >> 1));
    }
    return s;
}

// coordinates of the neighbour of x one step along mu (s = +1 or -1)
__device__ __forceinline__ void nb_coords(const Geom &g, const int x[4], int mu, int s, int y[4]) {
#pragma unroll
    for (int nu = 0; nu < 4; ++nu) y[nu] = x[nu];
    y[mu] = s > 0 ? (x[mu] == g.D[mu] - 1 ? 0 : x[mu] + 1) : (x[mu] == 0 ? g.D[mu] - 1 : x[mu] - 1);
}

// t = H_oe p_i at the odd entries (one entry per thread)
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_eo_hop(EP P) {
    typedef typename ArithT<S>::T R;
    const int N = P.nsite;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int i = st.inner_it;
        const R be = (R)st.beta.re;
        const bool first = (i == 0);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *pold = slot_cptr<S>((i & 1) ? P.p1 : P.pv, j, P.L);
        S *t = slot_ptr<S>(P.t, j, P.L);
        SITE_LOOP(0)
            int xc[4];
            const int s = half_site(P.g, 1, idx, xc);
            auto pn = [&](int y) -> R {
                const size_t h = (size_t)(y >> 1);
                R rv = ld_real(r, h);
                return first ? rv : rnd<S, R>(rv + be * (R)ld_real(pold, h));
            };
            R nb = R(0);
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                nb += pn(nb_fwd(P.g, s, xc, mu));
                nb += pn(nb_bwd(P.g, s, xc, mu));
            }
            st_real(t, (size_t)idx, nb);
        SITE_LOOP_END
    ITEM_LOOP_END
}

// p_i = r + beta p_{i-1} and q = S p_i = d p_i - H_eo t / d at the even
// entries; partial p_i . q
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_eo_apply(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32];
    const int N = P.nsite;
    const R diag = (R)P.diag, inv_d = (R)(1.0 / P.diag);
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int i = st.inner_it;
        const R be = (R)st.beta.re;
        const bool first = (i == 0);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *pold = slot_cptr<S>((i & 1) ? P.p1 : P.pv, j, P.L);
        const S *t = slot_cptr<S>(P.t, j, P.L);
        S *pnew = slot_ptr<S>((i & 1) ? P.pv : P.p1, j, P.L);
        S *q = slot_ptr<S>(P.q, j, P.L);
        R vr[1] = {R(0)};
        SITE_LOOP(0)
            int xc[4];
            const int s = half_site(P.g, 0, idx, xc);
            const R rv = ld_real(r, (size_t)idx);
            const R pc = first ? rv : rnd<S, R>(rv + be * (R)ld_real(pold, (size_t)idx));
            const R nb = half_nbsum<S, R>(P.g, t, s, xc);
            const R qv = rnd<S, R>(diag * pc - nb * inv_d);
            st_real(pnew, (size_t)idx, pc);
            st_real(q, (size_t)idx, qv);
            vr[0] += pc * qv;
        SITE_LOOP_END
        item_store_r<1>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

// Four half entries per thread (D_0 a multiple of 8, so that the quad
// h .. h+3, h a multiple of 4, lies in one x row and all four sites share
// their row parity b): the sites are s, s+2, s+4, s+6.  Their y, z, t
// neighbours are the aligned quad of the other parity at (neighbour of s) >> 1.
// With Q the other parity's quad at h, the +x / -x neighbours of entry k are
// Q[k] / Q[k-1] when b = 0 and Q[k+1] / Q[k] when b = 1; the one entry
// outside Q is a single load, wrapping within the row.  The neighbours are
// added in the one-entry kernels' order (x+, x-, y+, y-, z+, z-, t+, t-), so
// both paths give the same results.
template <typename S, typename R, typename F1, typename F4>
__device__ __forceinline__ void eo_nbsum4(const Geom &g, int h, int s, const int xc[4], F1 one, F4 quad,
                                          R acc[4]) {
    const int half_row = g.D[0] >> 1;
    const int c = (xc[0] - (s & 1)) >> 1;           // position of h in its row (multiple of 4)
    R Q[4], t4[4];
    quad(h, Q);
    if ((s & 1) == 0) {
        const R L = one(c == 0 ? h + half_row - 1 : h - 1);
        acc[0] = Q[0] + L; acc[1] = Q[1] + Q[0]; acc[2] = Q[2] + Q[1]; acc[3] = Q[3] + Q[2];
    } else {
        const R Rt = one(c + 4 == half_row ? h + 4 - half_row : h + 4);
        acc[0] = Q[1] + Q[0]; acc[1] = Q[2] + Q[1]; acc[2] = Q[3] + Q[2]; acc[3] = Rt + Q[3];
    }
#pragma unroll
    for (int mu = 1; mu < 4; ++mu) {
        quad(nb_fwd(g, s, xc, mu) >> 1, t4);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += t4[k];
        quad(nb_bwd(g, s, xc, mu) >> 1, t4);
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[k] += t4[k];
    }
}

template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_eo_hop_v4(EP P) {
    typedef typename ArithT<S>::T R;
    const int N = P.nsite;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int i = st.inner_it;
        const R be = (R)st.beta.re;
        const bool first = (i == 0);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *pold = slot_cptr<S>((i & 1) ? P.p1 : P.pv, j, P.L);
        S *t = slot_ptr<S>(P.t, j, P.L);
        QUAD_LOOP
            int xc[4];
            const int s = half_site(P.g, 1, idx, xc);
            auto pquad = [&](int h, R out[4]) {
                Quad<S>::ld(r, h, out);
                if (!first) {
                    R pp[4];
                    Quad<S>::ld(pold, h, pp);
#pragma unroll
                    for (int k = 0; k < 4; ++k) out[k] = rnd<S, R>(out[k] + be * pp[k]);
                }
            };
            auto pone = [&](int h) -> R {
                R rv = ld_real(r, (size_t)h);
                return first ? rv : rnd<S, R>(rv + be * (R)ld_real(pold, (size_t)h));
            };
            R acc[4];
            eo_nbsum4<S, R>(P.g, idx, s, xc, pone, pquad, acc);
            Quad<S>::st(t, idx, acc);
        QUAD_LOOP_END
    ITEM_LOOP_END
}

template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_eo_apply_v4(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32];
    const int N = P.nsite;
    const R diag = (R)P.diag, inv_d = (R)(1.0 / P.diag);
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int i = st.inner_it;
        const R be = (R)st.beta.re;
        const bool first = (i == 0);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *pold = slot_cptr<S>((i & 1) ? P.p1 : P.pv, j, P.L);
        const S *t = slot_cptr<S>(P.t, j, P.L);
        S *pnew = slot_ptr<S>((i & 1) ? P.pv : P.p1, j, P.L);
        S *q = slot_ptr<S>(P.q, j, P.L);
        R vr[1] = {R(0)};
        QUAD_LOOP
            int xc[4];
            const int s = half_site(P.g, 0, idx, xc);
            R pc[4], acc[4], qv[4];
            Quad<S>::ld(r, idx, pc);
            if (!first) {
                R pp[4];
                Quad<S>::ld(pold, idx, pp);
#pragma unroll
                for (int k = 0; k < 4; ++k) pc[k] = rnd<S, R>(pc[k] + be * pp[k]);
            }
            auto tone = [&](int h) -> R { return ld_real(t, (size_t)h); };
            auto tquad = [&](int h, R out[4]) { Quad<S>::ld(t, h, out); };
            eo_nbsum4<S, R>(P.g, idx, s, xc, tone, tquad, acc);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                qv[k] = rnd<S, R>(diag * pc[k] - acc[k] * inv_d);
                vr[0] += pc[k] * qv[k];
            }
            Quad<S>::st(pnew, idx, pc);
            Quad<S>::st(q, idx, qv);
        QUAD_LOOP_END
        item_store_r<1>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

// outer step, part 1: t64 = H_oe x64 at the odd entries (FP64); a new task
// starts from x = 0, so its t64 is zero (written, not hopped: the
// contraction reads it if the task converges at once)
__global__ void __launch_bounds__(PT_BLOCK) k_eo_outer_hop(EP P) {
    const int N = P.nsite;
    ITEM_LOOP(LIST_OUTER)
        const int ph = P.slots[j].phase;
        if (ph != PH_START && ph != PH_OUTER) continue;
        const double *x = P.x64 + (size_t)j * P.L;
        double *t = P.t64 + (size_t)j * P.L;
        if (ph == PH_START) {
            SITE_LOOP(0)
                t[idx] = 0.0;
            SITE_LOOP_END
            continue;
        }
        SITE_LOOP(0)
            int xc[4];
            const int s = half_site(P.g, 1, idx, xc);
            t[idx] = half_nbsum<double, double>(P.g, x, s, xc);
        SITE_LOOP_END
    ITEM_LOOP_END
}

// outer step, part 2, at the even entries: r64 = b'_e - S x64 in FP64, with
// b'_e = b_e + H_eo b_o / d formed from the regenerated source when the task
// starts (x = 0, so r64 = b'_e) and kept in FP64 for its later outer steps;
// r = (S) r64 starts the inner solve (e = 0).  Partials: |r64|^2, |b|^2 of
// both sites of the entry (even and odd; used when the task starts), |r|^2
// of the rounded r.
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_eo_outer_residual(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32 * 3];
    const int N = P.nsite;
    const double d = P.diag, inv_d = 1.0 / P.diag;
    ITEM_LOOP(LIST_OUTER)
        const Slot &st = P.slots[j];
        const int ph = st.phase;
        if (ph != PH_START && ph != PH_OUTER) continue;
        const Task tk = P.tasks[st.task];
        const uint64_t key = (P.mode == MODE_SOLVE) ? 0 : pt_set_key(P.seed, tk.set);
        S *r = slot_ptr<S>(P.r, j, P.L);
        S *e = slot_ptr<S>(P.e, j, P.L);
        const double *x = P.x64 + (size_t)j * P.L;
        const double *t = P.t64 + (size_t)j * P.L;
        double *bp = P.b64 + (size_t)j * P.L;
        // A probe's entries are 0 or +-1: their neighbour sum and |b|^2 are
        // exact in FP32 (user sources in solve mode stay FP64); |r|^2 of the
        // rounded r is summed in the inner solve's arithmetic.
        const bool probe = P.mode != MODE_SOLVE;
        double v0 = 0.0, v1d = 0.0;
        float v1f = 0.f;
        R v2r = R(0);
        SITE_LOOP(0)
            double rv;
            if (ph == PH_START) {
                int xc[4], y4[4];
                const int s = half_site(P.g, 0, idx, xc);
#pragma unroll
                for (int nu = 0; nu < 4; ++nu) y4[nu] = xc[nu];
                y4[0] ^= 1;                                  // the odd site of the same entry
                const Cx<double> be = source_val<0>(P, tk, key, s, xc, 0);
                const Cx<double> bo = source_val<0>(P, tk, key, s ^ 1, y4, 0);
                double b_nb;
                if (probe) {
                    float f = 0.f;
#pragma unroll
                    for (int mu = 0; mu < 4; ++mu) {
                        nb_coords(P.g, xc, mu, 1, y4);
                        f += (float)source_val<0>(P, tk, key, nb_fwd(P.g, s, xc, mu), y4, 0).re;
                        nb_coords(P.g, xc, mu, -1, y4);
                        f += (float)source_val<0>(P, tk, key, nb_bwd(P.g, s, xc, mu), y4, 0).re;
                    }
                    b_nb = (double)f;
                    v1f += (float)(be.re * be.re) + (float)(bo.re * bo.re);
                } else {
                    b_nb = 0.0;
#pragma unroll
                    for (int mu = 0; mu < 4; ++mu) {
                        nb_coords(P.g, xc, mu, 1, y4);
                        b_nb += source_val<0>(P, tk, key, nb_fwd(P.g, s, xc, mu), y4, 0).re;
                        nb_coords(P.g, xc, mu, -1, y4);
                        b_nb += source_val<0>(P, tk, key, nb_bwd(P.g, s, xc, mu), y4, 0).re;
                    }
                    v1d += be.re * be.re + bo.re * bo.re;
                }
                rv = be.re + b_nb * inv_d;                   // x = 0
                bp[idx] = rv;
            } else {
                int xc[4];
                const int s = half_site(P.g, 0, idx, xc);
                rv = bp[idx] - (d * x[idx] - half_nbsum<double, double>(P.g, t, s, xc) * inv_d);
            }
            v0 += rv * rv;
            const R rs = rnd<S, R>((R)rv);
            st_real(r, (size_t)idx, rs);
            st_real(e, (size_t)idx, R(0));
            v2r += rs * rs;
        SITE_LOOP_END
        double v[3] = {v0, v1d + (double)v1f, (double)v2r};
        item_store<3>(P, j, b, v, sh);
    ITEM_LOOP_END
}

// x at storage site y (coordinates xy): its even entry, or on an odd site
// x_o = (b_o + H_oe x_e) / d from the source and t64 = H_oe x_e, which the
// outer step formed for the final x_e (the slot converged right after it)
__device__ __forceinline__ double eo_x_at(const EP &P, const Task &tk, uint64_t key, const double *x,
                                          const double *t64, double inv_d, int y, const int xy[4]) {
    if (((xy[0] + xy[1] + xy[2] + xy[3]) & 1) == 0) return x[y >> 1];
    const double b_o = source_val<0>(P, tk, key, y, xy, 0).re;
    return (b_o + t64[y >> 1]) * inv_d;
}

// the contraction (trace mode) or the copy-out (solve mode) of k_contract for
// even-odd slots: entry h covers the sites 2h and 2h + 1
template <int MAXQ>
__global__ void __launch_bounds__(PT_BLOCK) k_eo_contract(EP P) {
    __shared__ double sh[32 * 2 * PT_MAX_P];
    const int N = P.nsite, NF = P.g.N;
    const double inv_d = 1.0 / P.diag;
    ITEM_LOOP(LIST_CONTRACT)
        const Slot &st = P.slots[j];
        if (st.phase != PH_CONTRACT) continue;
        const Task tk = P.tasks[st.task];
        const double *x = P.x64 + (size_t)j * P.L;
        const double *t64 = P.t64 + (size_t)j * P.L;
        const uint64_t key = (P.mode == MODE_SOLVE) ? 0 : pt_set_key(P.seed, tk.set);
        if (P.mode == MODE_SOLVE) {
            SITE_LOOP(0)
                for (int w = 0; w < 2; ++w) {
                    const int sw = 2 * idx + w;
                    int xs[4];
                    site_coords(P.g, sw, xs);
                    P.X_user[(size_t)tk.set * NF + sw] = eo_x_at(P, tk, key, x, t64, inv_d, sw, xs);
                }
            SITE_LOOP_END
            continue;
        }
        double acc[2 * MAXQ];
#pragma unroll
        for (int n = 0; n < 2 * MAXQ; ++n) acc[n] = 0.0;
        const int32_t *col = P.col + (size_t)tk.cidx * NF;
        SITE_LOOP(0)
            for (int w = 0; w < 2; ++w) {
                const int sw = 2 * idx + w;
                if (P.n_lev) {                 // the coarsest ancestor class holds every finer one
                    if (P.lev_cols[sw] != P.lev_anc[tk.colour]) continue;
                } else if (col[sw] != tk.colour) {
                    continue;
                }
                int xs[4], xy[4];
                site_coords(P.g, sw, xs);
                const Cx<double> z = pt_noise(key, (uint64_t)sw, P.noise);
#pragma unroll
                for (int n = 0; n < MAXQ; ++n) {
                    if (n >= P.n_p) break;
                    if (P.n_lev) {
                        const int l = n / P.n_pr;
                        if (l > 0 && P.lev_cols[(size_t)l * NF + sw] != P.lev_anc[(size_t)l * P.m_fin + tk.colour])
                            continue;
                    }
                    int cm;
                    const int y = shift_fwd(P.g, sw, xs, P.mu, P.p[n], &cm);
#pragma unroll
                    for (int nu = 0; nu < 4; ++nu) xy[nu] = xs[nu];
                    xy[P.mu] = cm;
                    const double xv = eo_x_at(P, tk, key, x, t64, inv_d, y, xy);
                    acc[2 * n] += z.re * xv;                // conj(z) x
                    acc[2 * n + 1] -= z.im * xv;
                }
            }
        SITE_LOOP_END
        item_store_contract<MAXQ>(P, j, b, acc, 2 * P.n_p, sh);
    ITEM_LOOP_END
}

// ------------------------------------------------------------------ BiCGStab (Wilson)
#ifndef PT_WIL_MINB
#define PT_WIL_MINB 3    // resident CTAs per SM the FP32/BF16 Wilson applies are compiled for
#endif
// v = A p;  partial (r0, v)
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BLOCK, std::is_same<S, double>::value ? 2 : PT_WIL_MINB) k_bicg_apply1(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 2];
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const S *pv = slot_cptr<S>(P.pv, j, P.L);
        S *q = slot_ptr<S>(P.q, j, P.L);
        const S *r0 = slot_cptr<S>(P.r0, j, P.L);
        R vr[2] = {R(0), R(0)};
        SITE_LOOP(1)
            int xc[4];
            site_coords(P.g, idx, xc);
            Cx<R> av[12];
            apply_site<1, R, S, LS>(P, pv, (const LS *)P.U, idx, xc, av);
            Cx<R> z[4][3];
            load_spinor<S, R>(r0, N, idx, z);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                av[c] = Cx<R>{rnd<S, R>(av[c].re), rnd<S, R>(av[c].im)};
                const Cx<R> w = av[c], zc = z[c / 3][c % 3];
                vr[0] += zc.re * w.re + zc.im * w.im;
                vr[1] += zc.re * w.im - zc.im * w.re;
            }
            store_spinor<S, R>(q, N, idx, av);
        SITE_LOOP_END
        item_store_r<2>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

__global__ void k_fin_bicg_alpha(EP P) {
    WARP_LOOP(LIST_INNER)
        if (st.phase != PH_INNER) continue;
        double tot[2];
        warp_total<2>(P, j, tot);
        if (lane == 0) {
            const double d2 = tot[0] * tot[0] + tot[1] * tot[1];
            if (!(d2 > 0.0) || !isfinite(d2)) {
                atomicOr(&P.flags[FLAG_NUMERIC], 4);
                st.phase = PH_OUTER;
            } else {  // alpha = rho / (r0, v)
                st.alpha = Cx<double>{(st.rho.re * tot[0] + st.rho.im * tot[1]) / d2,
                                      (st.rho.im * tot[0] - st.rho.re * tot[1]) / d2};
            }
        }
    WARP_LOOP_END
}

// s = r - alpha v
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_bicg_s(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    const int N = P.nsite;            // field entries per slot (N/2 in even-odd mode)
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const Cx<R> al = Cx<R>{(R)st.alpha.re, (R)st.alpha.im};
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *q = slot_cptr<S>(P.q, j, P.L);
        S *s = slot_ptr<S>(P.s, j, P.L);
        SITE_LOOP(1)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                Cx<R> rv[2], qv[2], sv[2];
                ld_pair<S, R>(r, N, k, idx, rv);
                ld_pair<S, R>(q, N, k, idx, qv);
                sv[0] = csub(rv[0], cmul(al, qv[0]));
                sv[1] = csub(rv[1], cmul(al, qv[1]));
                st_pair<S, R>(s, N, k, idx, sv);
            }
        SITE_LOOP_END
    ITEM_LOOP_END
}

// t = A s;  partials (t, s), |t|^2
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BLOCK, std::is_same<S, double>::value ? 2 : PT_WIL_MINB) k_bicg_apply2(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 3];
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const S *s = slot_cptr<S>(P.s, j, P.L);
        S *t = slot_ptr<S>(P.t, j, P.L);
        R vr[3] = {R(0), R(0), R(0)};
        SITE_LOOP(1)
            int xc[4];
            site_coords(P.g, idx, xc);
            Cx<R> acc[4][3], sp[4][3], av[12];
            wilson_hop_site<R, S, LS>(P.g, s, (const LS *)P.U, P.antip, idx, xc, acc);
            load_spinor<S, R>(s, N, idx, sp);                  // the own spinor, loaded once
            const R kap = (R)P.kappa;
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                const Cx<R> w = csub(sp[c / 3][c % 3], cscale(acc[c / 3][c % 3], kap));
                av[c] = Cx<R>{rnd<S, R>(w.re), rnd<S, R>(w.im)};
            }
            store_spinor<S, R>(t, N, idx, av);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                const Cx<R> tv = av[c];
                const Cx<R> sv = sp[c / 3][c % 3];
                vr[0] += tv.re * sv.re + tv.im * sv.im;     // (t, s) = conj(t) s
                vr[1] += tv.re * sv.im - tv.im * sv.re;
                vr[2] += tv.re * tv.re + tv.im * tv.im;
            }
        SITE_LOOP_END
        item_store_r<3>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

// Two right-hand sides per item (rhs_block = 2): the items pair consecutive
// entries of the work list, site block by site block within slot groups of
// max(1, gs / 2) pairs; every link is loaded once per site for both.  A pair
// whose second slot is missing or not iterating computes the first twice and
// keeps one result.
#define ITEM2_LOOP(LIST)                                                        \
    const int cnt = P.counts[LIST];                                             \
    const int *lst = P.lists + (size_t)(LIST) * P.R;                            \
    const int npairs_ = (cnt + 1) / 2;                                          \
    const int gp_ = max(1, P.gs / 2);                                           \
    const int64_t n_items = (int64_t)npairs_ * P.nsb;                           \
    const int64_t gitems_ = (int64_t)gp_ * P.nsb;                               \
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {              \
        const int64_t g_ = it / gitems_;                                        \
        const int base_ = (int)(g_ * gp_);                                      \
        const int gsz_ = min(gp_, npairs_ - base_);                             \
        const int rem_ = (int)(it - g_ * gitems_);                              \
        const int b = rem_ / gsz_;                                              \
        const int q_ = base_ + rem_ % gsz_;                                     \
        const int ja = lst[2 * q_];                                             \
        const int jb = (2 * q_ + 1 < cnt) ? lst[2 * q_ + 1] : -1;
#define ITEM2_LOOP_END }

// v = A p for two slots;  partials (r0, v) of each
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BLOCK, 2) k_bicg_apply1_x2(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 2];
    const int N = P.g.N;
    ITEM2_LOOP(LIST_INNER)
        const bool act_a = P.slots[ja].phase == PH_INNER;
        const bool act_b = jb >= 0 && P.slots[jb].phase == PH_INNER;
        if (!act_a && !act_b) continue;
        const int j0 = act_a ? ja : jb, j1 = (act_a && act_b) ? jb : j0;
        const S *const pv[2] = {slot_cptr<S>(P.pv, j0, P.L), slot_cptr<S>(P.pv, j1, P.L)};
        S *const q[2] = {slot_ptr<S>(P.q, j0, P.L), slot_ptr<S>(P.q, j1, P.L)};
        const S *const r0[2] = {slot_cptr<S>(P.r0, j0, P.L), slot_cptr<S>(P.r0, j1, P.L)};
        R vr[2][2] = {{R(0), R(0)}, {R(0), R(0)}};
        SITE_LOOP(1)
            int xc[4];
            site_coords(P.g, idx, xc);
            Cx<R> acc[2][4][3];
            wilson_hop_multi<R, S, LS, 2>(P.g, pv, (const LS *)P.U, P.antip, idx, xc, acc);
            const R kap = (R)P.kappa;
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                Cx<R> ps[4][3], z[4][3], av[12];
                load_spinor<S, R>(pv[n], N, idx, ps);
                load_spinor<S, R>(r0[n], N, idx, z);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const Cx<R> w = csub(ps[c / 3][c % 3], cscale(acc[n][c / 3][c % 3], kap));
                    av[c] = Cx<R>{rnd<S, R>(w.re), rnd<S, R>(w.im)};
                    const Cx<R> zc = z[c / 3][c % 3];
                    vr[n][0] += zc.re * av[c].re + zc.im * av[c].im;
                    vr[n][1] += zc.re * av[c].im - zc.im * av[c].re;
                }
                if (n == 0 || j1 != j0) store_spinor<S, R>(q[n], N, idx, av);
            }
        SITE_LOOP_END
        item_store_r<2>(P, j0, b, vr[0], sh);
        if (j1 != j0) item_store_r<2>(P, j1, b, vr[1], sh);
    ITEM2_LOOP_END
}

// t = A s for two slots;  partials (t, s), |t|^2 of each
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BLOCK, 2) k_bicg_apply2_x2(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 3];
    const int N = P.g.N;
    ITEM2_LOOP(LIST_INNER)
        const bool act_a = P.slots[ja].phase == PH_INNER;
        const bool act_b = jb >= 0 && P.slots[jb].phase == PH_INNER;
        if (!act_a && !act_b) continue;
        const int j0 = act_a ? ja : jb, j1 = (act_a && act_b) ? jb : j0;
        const S *const sv_[2] = {slot_cptr<S>(P.s, j0, P.L), slot_cptr<S>(P.s, j1, P.L)};
        S *const t[2] = {slot_ptr<S>(P.t, j0, P.L), slot_ptr<S>(P.t, j1, P.L)};
        R vr[2][3] = {{R(0), R(0), R(0)}, {R(0), R(0), R(0)}};
        SITE_LOOP(1)
            int xc[4];
            site_coords(P.g, idx, xc);
            Cx<R> acc[2][4][3];
            wilson_hop_multi<R, S, LS, 2>(P.g, sv_, (const LS *)P.U, P.antip, idx, xc, acc);
            const R kap = (R)P.kappa;
#pragma unroll
            for (int n = 0; n < 2; ++n) {
                Cx<R> sp[4][3], av[12];
                load_spinor<S, R>(sv_[n], N, idx, sp);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const Cx<R> w = csub(sp[c / 3][c % 3], cscale(acc[n][c / 3][c % 3], kap));
                    av[c] = Cx<R>{rnd<S, R>(w.re), rnd<S, R>(w.im)};
                    const Cx<R> tv = av[c], sc = sp[c / 3][c % 3];
                    vr[n][0] += tv.re * sc.re + tv.im * sc.im;
                    vr[n][1] += tv.re * sc.im - tv.im * sc.re;
                    vr[n][2] += tv.re * tv.re + tv.im * tv.im;
                }
                if (n == 0 || j1 != j0) store_spinor<S, R>(t[n], N, idx, av);
            }
        SITE_LOOP_END
        item_store_r<3>(P, j0, b, vr[0], sh);
        if (j1 != j0) item_store_r<3>(P, j1, b, vr[1], sh);
    ITEM2_LOOP_END
}

__global__ void k_fin_bicg_omega(EP P) {
    WARP_LOOP(LIST_INNER)
        if (st.phase != PH_INNER) continue;
        double tot[3];
        warp_total<3>(P, j, tot);
        if (lane == 0) {
            if (!(tot[2] > 0.0) || !isfinite(tot[2])) st.omega = Cx<double>{0.0, 0.0};
            else st.omega = Cx<double>{tot[0] / tot[2], tot[1] / tot[2]};
        }
    WARP_LOOP_END
}

// e += alpha p + omega s;  r = s - omega t;  partials (r0, r), |r|^2
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_bicg_update(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 3];
    const int N = P.nsite;            // field entries per slot (N/2 in even-odd mode)
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const Cx<R> al = Cx<R>{(R)st.alpha.re, (R)st.alpha.im};
        const Cx<R> om = Cx<R>{(R)st.omega.re, (R)st.omega.im};
        S *e = slot_ptr<S>(P.e, j, P.L);
        S *r = slot_ptr<S>(P.r, j, P.L);
        const S *pv = slot_cptr<S>(P.pv, j, P.L);
        const S *s = slot_cptr<S>(P.s, j, P.L);
        const S *t = slot_cptr<S>(P.t, j, P.L);
        const S *r0 = slot_cptr<S>(P.r0, j, P.L);
        R vr[3] = {R(0), R(0), R(0)};
        SITE_LOOP(1)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                Cx<R> sv[2], ev[2], pp[2], tv[2], zv[2], rv[2];
                ld_pair<S, R>(s, N, k, idx, sv);
                ld_pair<S, R>(e, N, k, idx, ev);
                ld_pair<S, R>(pv, N, k, idx, pp);
                ld_pair<S, R>(t, N, k, idx, tv);
                ld_pair<S, R>(r0, N, k, idx, zv);
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    ev[h] = cadd(ev[h], cadd(cmul(al, pp[h]), cmul(om, sv[h])));
                    const Cx<R> rv0 = csub(sv[h], cmul(om, tv[h]));
                    rv[h] = Cx<R>{rnd<S, R>(rv0.re), rnd<S, R>(rv0.im)};
                    vr[0] += zv[h].re * rv[h].re + zv[h].im * rv[h].im;
                    vr[1] += zv[h].re * rv[h].im - zv[h].im * rv[h].re;
                    vr[2] += rv[h].re * rv[h].re + rv[h].im * rv[h].im;
                }
                st_pair<S, R>(e, N, k, idx, ev);
                st_pair<S, R>(r, N, k, idx, rv);
            }
        SITE_LOOP_END
        item_store_r<3>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

__global__ void k_fin_bicg_beta(EP P) {
    WARP_LOOP(LIST_INNER)
        if (st.phase != PH_INNER) continue;
        double tot[3];
        warp_total<3>(P, j, tot);
        if (lane == 0) {
            st.inner_it += 1;
            st.total_it += 1;
            const double om2 = st.omega.re * st.omega.re + st.omega.im * st.omega.im;
            const double rho2 = st.rho.re * st.rho.re + st.rho.im * st.rho.im;
            if (tot[2] <= st.target2 || st.inner_it >= P.max_inner || st.total_it >= P.maxit ||
                !isfinite(tot[2]) || !(om2 > 0.0) || !(rho2 > 0.0)) {
                st.phase = PH_OUTER;
            } else {  // beta = (rho' / rho) (alpha / omega)
                const Cx<double> rn = Cx<double>{tot[0], tot[1]};
                const Cx<double> q1 = Cx<double>{(rn.re * st.rho.re + rn.im * st.rho.im) / rho2,
                                                 (rn.im * st.rho.re - rn.re * st.rho.im) / rho2};
                const Cx<double> q2 = Cx<double>{(st.alpha.re * st.omega.re + st.alpha.im * st.omega.im) / om2,
                                                 (st.alpha.im * st.omega.re - st.alpha.re * st.omega.im) / om2};
                st.beta = cmul(q1, q2);
                st.rho = rn;
                st.rr = tot[2];
            }
        }
    WARP_LOOP_END
}

// p = r + beta (p - omega v)
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_bicg_dir(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    const int N = P.nsite;            // field entries per slot (N/2 in even-odd mode)
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const Cx<R> be = Cx<R>{(R)st.beta.re, (R)st.beta.im};
        const Cx<R> om = Cx<R>{(R)st.omega.re, (R)st.omega.im};
        S *pv = slot_ptr<S>(P.pv, j, P.L);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *q = slot_cptr<S>(P.q, j, P.L);
        SITE_LOOP(1)
#pragma unroll
            for (int k = 0; k < 6; ++k) {
                Cx<R> pp[2], qv[2], rv[2];
                ld_pair<S, R>(pv, N, k, idx, pp);
                ld_pair<S, R>(q, N, k, idx, qv);
                ld_pair<S, R>(r, N, k, idx, rv);
                pp[0] = cadd(rv[0], cmul(be, csub(pp[0], cmul(om, qv[0]))));
                pp[1] = cadd(rv[1], cmul(be, csub(pp[1], cmul(om, qv[1]))));
                st_pair<S, R>(pv, N, k, idx, pp);
            }
        SITE_LOOP_END
    ITEM_LOOP_END
}

// ------------------------------------------------------------------ even-odd link order
// A packed link array is chunk-major: chunk c of site s at c * N + s (FP32:
// five 16-byte chunks per direction; FP64 and BF16: one complex entry per
// chunk, nine per direction).
template <typename LS> struct LinkLayout;
template <> struct LinkLayout<float> { typedef float4 E; static constexpr int CHUNKS = 20; };
template <> struct LinkLayout<double> { typedef double2 E; static constexpr int CHUNKS = 36; };
template <> struct LinkLayout<__nv_bfloat16> { typedef uint32_t E; static constexpr int CHUNKS = 36; };

// the even-odd ordered copy: chunk c of site s (parity par) moves to
// c * N + par * N/2 + s/2; nothing else changes, so a kernel reading the
// copy at that position gets the same link bits
template <typename E>
__global__ void k_links_eo(Geom g, int n_chunk, const E *__restrict__ src, E *__restrict__ dst) {
    const int N = g.N;
    const int64_t total = (int64_t)n_chunk * N;
    for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = t / N;
        const int s = (int)(t - c * N);
        int r = s, par = 0;
        for (int d = 0; d < 4; ++d) {
            par += r % g.D[d];
            r /= g.D[d];
        }
        dst[c * N + (par & 1) * (N >> 1) + (s >> 1)] = src[t];
    }
}

// ------------------------------------------------------------------ even-odd BiCGStab (Wilson)
// With every side even, A = 1 - kappa D has D_ee = D_oo = 0, and A x = b is
// solved through the Schur complement on the even sites:
//   S x_e = b'_e,  S = 1 - kappa^2 D_eo D_oe,  b'_e = b_e + kappa D_eo b_o,
//   x_o = b_o + kappa D_oe x_e.
// Each application of S is two half-lattice hops: k_weo_hop forms
// h = D_oe p at the odd entries, k_weo_apply1 / k_weo_apply2 then p - kappa^2
// D_eo h at the even entries with BiCGStab's dot products.  S is better
// conditioned than A (about half the iterations) and its vectors are half as
// long.  The FP64 outer step forms t64 = D_oe x64 at the odd entries, then
// r = b'_e - S x64 at the even ones; b'_e is formed once per task (its first
// outer step, from the source regenerated at the site and its eight odd
// neighbours) and kept in FP64.  The stopping test is the full system's
// ||b - A x|| / ||b|| with |b|^2 over both parities (r_o = 0 once x_o is
// rebuilt).  The contraction and the copy-out read x_o = b_o + kappa t64,
// t64 = D_oe x64 of the final x64, where they read an odd site.
// With a clover term (A = A_W + C, diagonal blocks A_ee = 1 + C_ee and
// A_oo = 1 + C_oo) the same kernels form S = A_ee - kappa^2 D_eo A_oo^{-1}
// D_oe, b'_e = b_e + kappa D_eo A_oo^{-1} b_o and x_o = A_oo^{-1} (b_o +
// kappa D_oe x_e): the odd-site hops apply A_oo^{-1} before they store, the
// even-site applies A_ee to their own entry.

// One hop of the Wilson hopping term into acc at site idx (coordinates x):
// forward (1 - g_mu) U_mu(x) psi(x + mu) or backward (1 + g_mu)
// U_mu(x - mu)^dagger psi(x - mu), with psi = ps the neighbour's spinor and
// the boundary sign of antiperiodic time
template <typename R, typename LS>
__device__ __forceinline__ void wilson_hop_dir(const Geom &g, const LS *U, int antip, int idx, const int x[4],
                                               int mu, bool fwd, const Cx<R> ps[4][3], Cx<R> acc[4][3]) {
    Cx<R> h[2][3], uh[2][3], u[3][3];
    if (fwd) {
        const R eta = (antip && mu == 3 && x[3] == g.D[3] - 1) ? R(-1) : R(1);
        spin_project<R>(mu, R(-1), ps, h);
        load_link<R, LS>(U, g.N, mu, idx, u);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                Cx<R> t = cmul(u[a][0], h[k][0]);
                t = cadd(t, cmul(u[a][1], h[k][1]));
                t = cadd(t, cmul(u[a][2], h[k][2]));
                uh[k][a] = t;
            }
        spin_accumulate<R>(mu, R(-1), eta, uh, acc);
    } else {
        const R eta = (antip && mu == 3 && x[3] == 0) ? R(-1) : R(1);
        spin_project<R>(mu, R(1), ps, h);
        load_link<R, LS>(U, g.N, mu, nb_bwd(g, idx, x, mu), u);
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                Cx<R> t = cconjmul(u[0][a], h[k][0]);
                t = cadd(t, cconjmul(u[1][a], h[k][1]));
                t = cadd(t, cconjmul(u[2][a], h[k][2]));
                uh[k][a] = t;
            }
        spin_accumulate<R>(mu, R(1), eta, uh, acc);
    }
}

// position of the links of site s (parity par) in the even-odd ordered link
// copy of the inner solver: entry par * N/2 + s/2, its half-field entry, so
// that a warp of consecutive half entries reads consecutive links (in the
// full-lattice order the sites of one parity are two apart)
__device__ __forceinline__ int eo_link_pos(int N, int s, int par) { return par * (N >> 1) + (s >> 1); }
template <int LPAR>
__device__ __forceinline__ int link_pos(int N, int s, int par) {
    if constexpr (LPAR < 0) return s;
    else return eo_link_pos(N, s, par);
}

// (H psi)(x) at site idx (coordinates x) as in wilson_hop_site, with the
// neighbour spinors supplied by fetch(y, mu, dir, ps) (dir +1 forward, -1
// backward) and the links from a packed array in the full-lattice order
// (LPAR = -1) or in the even-odd order with idx of parity LPAR
template <typename R, typename LS, int LPAR = -1, typename Fetch>
__device__ __forceinline__ void wilson_hop_fetch(const Geom &g, Fetch fetch, const LS *U, int antip, int idx,
                                                 const int x[4], Cx<R> acc[4][3]) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[s][a] = Cx<R>{R(0), R(0)};
    const int N = g.N;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        {   // forward hop: (1 - g_mu) U_mu(x) psi(x + mu)
            const int y = nb_fwd(g, idx, x, mu);
            const R eta = (antip && mu == 3 && x[3] == g.D[3] - 1) ? R(-1) : R(1);
            Cx<R> ps[4][3], h[2][3], uh[2][3], u[3][3];
            fetch(y, mu, 1, ps);
            spin_project<R>(mu, R(-1), ps, h);
            load_link<R, LS>(U, N, mu, link_pos<LPAR>(N, idx, LPAR), u);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Cx<R> t = cmul(u[a][0], h[k][0]);
                    t = cadd(t, cmul(u[a][1], h[k][1]));
                    t = cadd(t, cmul(u[a][2], h[k][2]));
                    uh[k][a] = t;
                }
            spin_accumulate<R>(mu, R(-1), eta, uh, acc);
        }
        {   // backward hop: (1 + g_mu) U_mu(x - mu)^dagger psi(x - mu)
            const int y = nb_bwd(g, idx, x, mu);
            const R eta = (antip && mu == 3 && x[3] == 0) ? R(-1) : R(1);
            Cx<R> ps[4][3], h[2][3], uh[2][3], u[3][3];
            fetch(y, mu, -1, ps);
            spin_project<R>(mu, R(1), ps, h);
            load_link<R, LS>(U, N, mu, link_pos<LPAR>(N, y, 1 - LPAR), u);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Cx<R> t = cconjmul(u[0][a], h[k][0]);
                    t = cadd(t, cconjmul(u[1][a], h[k][1]));
                    t = cadd(t, cconjmul(u[2][a], h[k][2]));
                    uh[k][a] = t;
                }
            spin_accumulate<R>(mu, R(1), eta, uh, acc);
        }
    }
}

// whether the source of a task can be nonzero at storage site y: a probe
// lives on its colour class only (user sources in solve mode everywhere)
__device__ __forceinline__ bool source_may_be_nonzero(const EP &P, const Task &tk, int y) {
    if (P.mode == MODE_SOLVE || (tk.flags & TASK_ADJ)) return true;
    return P.col[(size_t)tk.cidx * P.g.N + y] == tk.colour;
}

// resident CTAs per SM the even-odd Wilson item kernels are compiled for:
// clv 0 plain, 1 a clover variant that fits the plain budget, 2 one that
// needs more registers per thread (FP64 storage: every clover variant)
template <typename S>
constexpr int weo_minb(int clv) {
    return std::is_same<S, double>::value ? (clv ? 1 : 2) : (clv == 2 ? 2 : PT_WIL_MINB);
}

// h = D_oe p at the odd entries (WHICH 0: p = pv, the first apply; 1: p = s);
// with the clover term (CLV) h = A_oo^{-1} D_oe p
template <typename S, typename LS, int WHICH, int CLV = 0>
__global__ void __launch_bounds__(PT_BLOCK, weo_minb<S>(CLV)) k_weo_hop(EP P) {
    typedef typename ArithT<S>::T R;
    const int N = P.nsite;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const S *src = slot_cptr<S>(WHICH ? P.s : P.pv, j, P.L);
        S *h = slot_ptr<S>(P.p1, j, P.L);
        SITE_LOOP(1)
            int xc[4];
            const int s = half_site(P.g, 1, idx, xc);
            Cx<R> acc[4][3], o[12];
            wilson_hop_fetch<R, LS, 1>(
                P.g, [&](int y, int, int, Cx<R> ps[4][3]) { load_spinor<S, R>(src, N, y >> 1, ps); },
                (const LS *)P.U, P.antip, s, xc, acc);
#pragma unroll
            for (int c = 0; c < 12; ++c) o[c] = acc[c / 3][c % 3];
            if constexpr (CLV) {
                if constexpr (std::is_same<S, double>::value) clover_mul(P.CL64, N, 1, idx, o);
                else clover_mul(P.CL32, N, 1, idx, o);
            }
#pragma unroll
            for (int c = 0; c < 12; ++c) o[c] = Cx<R>{rnd<S, R>(o[c].re), rnd<S, R>(o[c].im)};
            store_spinor<S, R>(h, N, idx, o);
        SITE_LOOP_END
    ITEM_LOOP_END
}

// v = S p = p - kappa^2 D_eo h at the even entries (clover: A_ee p - ...);
// partial (r0, v)
template <typename S, typename LS, int CLV = 0>
__global__ void __launch_bounds__(PT_BLOCK, weo_minb<S>(CLV)) k_weo_apply1(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32 * 2];
    const int N = P.nsite;
    const R k2 = (R)(P.kappa * P.kappa);
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const S *pv = slot_cptr<S>(P.pv, j, P.L);
        const S *h = slot_cptr<S>(P.p1, j, P.L);
        const S *r0 = slot_cptr<S>(P.r0, j, P.L);
        S *q = slot_ptr<S>(P.q, j, P.L);
        R vr[2] = {R(0), R(0)};
        SITE_LOOP(1)
            int xc[4];
            const int s = half_site(P.g, 0, idx, xc);
            Cx<R> acc[4][3], ps[4][3], z[4][3], av[12];
            wilson_hop_fetch<R, LS, 0>(
                P.g, [&](int y, int, int, Cx<R> f[4][3]) { load_spinor<S, R>(h, N, y >> 1, f); },
                (const LS *)P.U, P.antip, s, xc, acc);
            load_spinor<S, R>(pv, N, idx, ps);
            if constexpr (CLV) {
                Cx<R> v[12];
#pragma unroll
                for (int c = 0; c < 12; ++c) v[c] = ps[c / 3][c % 3];
                if constexpr (std::is_same<S, double>::value) clover_mul(P.CL64, N, 0, idx, v);
                else clover_mul(P.CL32, N, 0, idx, v);
#pragma unroll
                for (int c = 0; c < 12; ++c) ps[c / 3][c % 3] = v[c];
            }
            load_spinor<S, R>(r0, N, idx, z);
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                const Cx<R> w = csub(ps[c / 3][c % 3], cscale(acc[c / 3][c % 3], k2));
                av[c] = Cx<R>{rnd<S, R>(w.re), rnd<S, R>(w.im)};
                const Cx<R> zc = z[c / 3][c % 3];
                vr[0] += zc.re * av[c].re + zc.im * av[c].im;
                vr[1] += zc.re * av[c].im - zc.im * av[c].re;
            }
            store_spinor<S, R>(q, N, idx, av);
        SITE_LOOP_END
        item_store_r<2>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

// t = S s = s - kappa^2 D_eo h at the even entries (clover: A_ee s - ...);
// partials (t, s), |t|^2
template <typename S, typename LS, int CLV = 0>
__global__ void __launch_bounds__(PT_BLOCK, weo_minb<S>(2 * CLV)) k_weo_apply2(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32 * 3];
    const int N = P.nsite;
    const R k2 = (R)(P.kappa * P.kappa);
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const S *sv = slot_cptr<S>(P.s, j, P.L);
        const S *h = slot_cptr<S>(P.p1, j, P.L);
        S *t = slot_ptr<S>(P.t, j, P.L);
        R vr[3] = {R(0), R(0), R(0)};
        SITE_LOOP(1)
            int xc[4];
            const int s = half_site(P.g, 0, idx, xc);
            Cx<R> acc[4][3], sp[4][3], av[12];
            wilson_hop_fetch<R, LS, 0>(
                P.g, [&](int y, int, int, Cx<R> f[4][3]) { load_spinor<S, R>(h, N, y >> 1, f); },
                (const LS *)P.U, P.antip, s, xc, acc);
            if constexpr (CLV) {
                Cx<R> v[12];
                {
                    Cx<R> f[4][3];
                    load_spinor<S, R>(sv, N, idx, f);
#pragma unroll
                    for (int c = 0; c < 12; ++c) v[c] = f[c / 3][c % 3];
                }
                if constexpr (std::is_same<S, double>::value) clover_mul(P.CL64, N, 0, idx, v);
                else clover_mul(P.CL32, N, 0, idx, v);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const Cx<R> w = csub(v[c], cscale(acc[c / 3][c % 3], k2));
                    av[c] = Cx<R>{rnd<S, R>(w.re), rnd<S, R>(w.im)};
                }
                store_spinor<S, R>(t, N, idx, av);
                load_spinor<S, R>(sv, N, idx, sp);           // s itself, for the dot products
            } else {
                load_spinor<S, R>(sv, N, idx, sp);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const Cx<R> w = csub(sp[c / 3][c % 3], cscale(acc[c / 3][c % 3], k2));
                    av[c] = Cx<R>{rnd<S, R>(w.re), rnd<S, R>(w.im)};
                }
                store_spinor<S, R>(t, N, idx, av);
            }
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                const Cx<R> tv = av[c], sc = sp[c / 3][c % 3];
                vr[0] += tv.re * sc.re + tv.im * sc.im;     // (t, s) = conj(t) s
                vr[1] += tv.re * sc.im - tv.im * sc.re;
                vr[2] += tv.re * tv.re + tv.im * tv.im;
            }
        SITE_LOOP_END
        item_store_r<3>(P, j, b, vr, sh);
    ITEM_LOOP_END
}

// outer step, part 1: t64 = D_oe x64 at the odd entries (FP64); a new task
// starts from x = 0, so its t64 is zero (written, not hopped: the
// contraction reads it if the task converges at once)
__global__ void __launch_bounds__(PT_BLOCK) k_weo_outer_hop(EP P) {
    const int N = P.nsite;
    ITEM_LOOP(LIST_OUTER)
        const int ph = P.slots[j].phase;
        if (ph != PH_START && ph != PH_OUTER) continue;
        const double *x = P.x64 + (size_t)j * P.L;
        double *t = P.t64 + (size_t)j * P.L;
        SITE_LOOP(1)
            Cx<double> o[12];
            if (ph == PH_START) {
#pragma unroll
                for (int c = 0; c < 12; ++c) o[c] = Cx<double>{0.0, 0.0};
            } else {
                int xc[4];
                const int s = half_site(P.g, 1, idx, xc);
                Cx<double> acc[4][3];
                wilson_hop_fetch<double, double>(
                    P.g, [&](int y, int, int, Cx<double> f[4][3]) { load_spinor<double, double>(x, N, y >> 1, f); },
                    P.U64, P.antip, s, xc, acc);
#pragma unroll
                for (int c = 0; c < 12; ++c) o[c] = acc[c / 3][c % 3];
                if (P.clover) clover_mul(P.CL64, N, 1, idx, o);      // t64 = A_oo^{-1} D_oe x64
            }
            store_spinor<double, double>(t, N, idx, o);
        SITE_LOOP_END
    ITEM_LOOP_END
}

// outer step, part 2 (new tasks only), at the even entries: b'_e = b_e +
// kappa D_eo b_o from the source regenerated at the site and at those of its
// eight odd neighbours where it can be nonzero (a skipped neighbour would add
// exact zeros); kept in FP64 for the task's later outer steps
__global__ void __launch_bounds__(PT_BLOCK) k_weo_outer_bprime(EP P) {
    const int N = P.nsite;
    const double kap = P.kappa;
    ITEM_LOOP(LIST_OUTER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_START) continue;
        const Task tk = P.tasks[st.task];
        const uint64_t key = (P.mode == MODE_SOLVE) ? 0 : pt_set_key(P.seed, tk.set);
        double *bp = P.b64 + (size_t)j * P.L;
        SITE_LOOP(1)
            int xc[4];
            const int s = half_site(P.g, 0, idx, xc);
            Cx<double> acc[4][3], bv[12];
#pragma unroll
            for (int sp = 0; sp < 4; ++sp)
#pragma unroll
                for (int a = 0; a < 3; ++a) acc[sp][a] = Cx<double>{0.0, 0.0};
#pragma unroll
            for (int mu = 0; mu < 4; ++mu)
#pragma unroll
                for (int dir = 1; dir >= -1; dir -= 2) {
                    const int y = dir > 0 ? nb_fwd(P.g, s, xc, mu) : nb_bwd(P.g, s, xc, mu);
                    if (!source_may_be_nonzero(P, tk, y)) continue;
                    int y4[4];
                    nb_coords(P.g, xc, mu, dir, y4);
                    Cx<double> f[4][3];
                    if (P.clover) {                           // A_oo^{-1} b_o at the neighbour
                        Cx<double> v[12];
#pragma unroll
                        for (int c = 0; c < 12; ++c) v[c] = source_val<1>(P, tk, key, y, y4, c);
                        clover_mul(P.CL64, N, 1, y >> 1, v);
#pragma unroll
                        for (int c = 0; c < 12; ++c) f[c / 3][c % 3] = v[c];
                    } else {
#pragma unroll
                        for (int c = 0; c < 12; ++c) f[c / 3][c % 3] = source_val<1>(P, tk, key, y, y4, c);
                    }
                    wilson_hop_dir<double, double>(P.g, P.U64, P.antip, s, xc, mu, dir > 0, f, acc);
                }
#pragma unroll
            for (int c = 0; c < 12; ++c)
                bv[c] = cadd(source_val<1>(P, tk, key, s, xc, c), cscale(acc[c / 3][c % 3], kap));
            store_spinor<double, double>(bp, N, idx, bv);
        SITE_LOOP_END
    ITEM_LOOP_END
}

// outer step, part 3, at the even entries: r64 = b'_e - S x64 in FP64
// (= b'_e for a new task, x = 0); r = (S) r64 starts the inner solve
// (p = r0 = r, e = 0).  Partials: |r64|^2, |b|^2 of both sites of the entry
// (even and odd; used when the task starts), |r|^2 of the rounded r.
template <typename S>
__global__ void __launch_bounds__(PT_BLOCK) k_weo_outer_residual(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ double sh[32 * 3];
    const int N = P.nsite;
    const double k2 = P.kappa * P.kappa;
    ITEM_LOOP(LIST_OUTER)
        const Slot &st = P.slots[j];
        const int ph = st.phase;
        if (ph != PH_START && ph != PH_OUTER) continue;
        const Task tk = P.tasks[st.task];
        const uint64_t key = (P.mode == MODE_SOLVE) ? 0 : pt_set_key(P.seed, tk.set);
        S *r = slot_ptr<S>(P.r, j, P.L);
        S *pv = slot_ptr<S>(P.pv, j, P.L);
        S *r0 = slot_ptr<S>(P.r0, j, P.L);
        S *e = slot_ptr<S>(P.e, j, P.L);
        const double *x = P.x64 + (size_t)j * P.L;
        const double *t = P.t64 + (size_t)j * P.L;
        const double *bp = P.b64 + (size_t)j * P.L;
        double v[3] = {0.0, 0.0, 0.0};
        SITE_LOOP(1)
            int xc[4];
            const int s = half_site(P.g, 0, idx, xc);
            Cx<double> rv[12];
            if (ph == PH_START) {
                int xp[4] = {xc[0] ^ 1, xc[1], xc[2], xc[3]};          // the odd site of the same entry
                Cx<double> bs[4][3];
                load_spinor<double, double>(bp, N, idx, bs);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const Cx<double> be = source_val<1>(P, tk, key, s, xc, c);
                    const Cx<double> bo = source_val<1>(P, tk, key, s ^ 1, xp, c);
                    v[1] += be.re * be.re + be.im * be.im + bo.re * bo.re + bo.im * bo.im;
                    rv[c] = bs[c / 3][c % 3];                           // x = 0
                }
            } else {
                Cx<double> acc[4][3];
                wilson_hop_fetch<double, double>(
                    P.g, [&](int y, int, int, Cx<double> f[4][3]) { load_spinor<double, double>(t, N, y >> 1, f); },
                    P.U64, P.antip, s, xc, acc);
                if (P.clover) {
                    // r = b' - A_ee x + kappa^2 D_eo t64
                    Cx<double> xv[12];
#pragma unroll
                    for (int c = 0; c < 12; ++c) xv[c] = ld_cx<double, double>(x, N, c, idx);
                    clover_mul(P.CL64, N, 0, idx, xv);
#pragma unroll
                    for (int c = 0; c < 12; ++c)
                        rv[c] = csub(ld_cx<double, double>(bp, N, c, idx), csub(xv[c], cscale(acc[c / 3][c % 3], k2)));
                } else {
                    // r = b' - x + kappa^2 D_eo t64, component by component
#pragma unroll
                    for (int c = 0; c < 12; ++c) {
                        const Cx<double> bc = ld_cx<double, double>(bp, N, c, idx);
                        const Cx<double> xcc = ld_cx<double, double>(x, N, c, idx);
                        rv[c] = csub(bc, csub(xcc, cscale(acc[c / 3][c % 3], k2)));
                    }
                }
            }
            Cx<R> rs[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                v[0] += rv[c].re * rv[c].re + rv[c].im * rv[c].im;
                rs[c] = Cx<R>{rnd<S, R>((R)rv[c].re), rnd<S, R>((R)rv[c].im)};
                v[2] += (double)rs[c].re * (double)rs[c].re + (double)rs[c].im * (double)rs[c].im;
            }
            store_spinor<S, R>(r, N, idx, rs);
            store_spinor<S, R>(pv, N, idx, rs);
            store_spinor<S, R>(r0, N, idx, rs);
            Cx<R> zero[12];
#pragma unroll
            for (int c = 0; c < 12; ++c) zero[c] = Cx<R>{R(0), R(0)};
            store_spinor<S, R>(e, N, idx, zero);
        SITE_LOOP_END
        item_store<3>(P, j, b, v, sh);
    ITEM_LOOP_END
}

// x at storage site y (coordinates xy), all 12 components: its even entry,
// or on an odd site x_o = b_o + kappa D_oe x_e from the source and
// t64 = D_oe x_e, which the outer step formed for the final x_e (zero for a
// task that converged at its first step, where x = 0); with the clover term
// x_o = A_oo^{-1} b_o + kappa t64, t64 = A_oo^{-1} D_oe x_e
__device__ __forceinline__ void weo_x_at(const EP &P, const Task &tk, uint64_t key, const double *x,
                                         const double *t64, int y, const int xy[4], Cx<double> out[12]) {
    const int N = P.nsite;
    Cx<double> f[4][3];
    if (((xy[0] + xy[1] + xy[2] + xy[3]) & 1) == 0) {
        load_spinor<double, double>(x, N, y >> 1, f);
#pragma unroll
        for (int c = 0; c < 12; ++c) out[c] = f[c / 3][c % 3];
        return;
    }
    load_spinor<double, double>(t64, N, y >> 1, f);
    Cx<double> bo[12];
#pragma unroll
    for (int c = 0; c < 12; ++c) bo[c] = source_val<1>(P, tk, key, y, xy, c);
    if (P.clover && source_may_be_nonzero(P, tk, y)) clover_mul(P.CL64, N, 1, y >> 1, bo);   // A_oo^{-1} b_o
#pragma unroll
    for (int c = 0; c < 12; ++c) out[c] = cadd(bo[c], cscale(f[c / 3][c % 3], P.kappa));
}

// the contraction (trace mode) or the copy-out (solve mode) for even-odd
// Wilson slots: entry h covers the sites 2h and 2h + 1
template <int MAXQ>
__global__ void __launch_bounds__(PT_BLOCK) k_weo_contract(EP P) {
    __shared__ double sh[32 * 2 * PT_MAX_P];
    const int N = P.nsite, NF = P.g.N;
    ITEM_LOOP(LIST_CONTRACT)
        const Slot &st = P.slots[j];
        if (st.phase != PH_CONTRACT) continue;
        const Task tk = P.tasks[st.task];
        const double *x = P.x64 + (size_t)j * P.L;
        const double *t64 = P.t64 + (size_t)j * P.L;
        const uint64_t key = (P.mode == MODE_SOLVE) ? 0 : pt_set_key(P.seed, tk.set);
        if (P.mode == MODE_SOLVE) {
            SITE_LOOP(1)
                for (int w = 0; w < 2; ++w) {
                    const int sw = 2 * idx + w;
                    int xs[4];
                    site_coords(P.g, sw, xs);
                    Cx<double> xv[12];
                    weo_x_at(P, tk, key, x, t64, sw, xs, xv);
                    double *dst = P.X_user + ((size_t)tk.set * NF + sw) * 24;
                    for (int c = 0; c < 12; ++c) {
                        dst[2 * c] = xv[c].re;
                        dst[2 * c + 1] = xv[c].im;
                    }
                }
            SITE_LOOP_END
            continue;
        }
        double acc[2 * MAXQ];
#pragma unroll
        for (int n = 0; n < 2 * MAXQ; ++n) acc[n] = 0.0;
        const int32_t *col = P.col + (size_t)tk.cidx * NF;
        SITE_LOOP(1)
            for (int w = 0; w < 2; ++w) {
                const int sw = 2 * idx + w;
                if (P.n_lev) {                 // the coarsest ancestor class holds every finer one
                    if (P.lev_cols[sw] != P.lev_anc[tk.colour]) continue;
                } else if (col[sw] != tk.colour) {
                    continue;
                }
                int xs[4], xy[4];
                site_coords(P.g, sw, xs);
                for (int n = 0; n < MAXQ; ++n) {
                    if (n >= P.n_p) break;
                    if (P.n_lev) {
                        const int l = n / P.n_pr;
                        if (l > 0 && P.lev_cols[(size_t)l * NF + sw] != P.lev_anc[(size_t)l * P.m_fin + tk.colour])
                            continue;
                    }
                    int cm;
                    const int y = shift_fwd(P.g, sw, xs, P.mu, P.p[n], &cm);
                    for (int nu = 0; nu < 4; ++nu) xy[nu] = xs[nu];
                    xy[P.mu] = cm;
                    Cx<double> xv[12];
                    weo_x_at(P, tk, key, x, t64, y, xy, xv);
                    for (int a = 0; a < 12; ++a) {
                        if (P.dilute && a != tk.comp) continue;
                        const Cx<double> z = P.dilute ? pt_noise(key, (uint64_t)sw, P.noise)
                                                      : pt_noise(key, (uint64_t)sw * 12 + a, P.noise);
                        const Cx<double> q = cconjmul(z, xv[a]);
                        acc[2 * n] += q.re;
                        acc[2 * n + 1] += q.im;
                    }
                }
            }
        SITE_LOOP_END
        item_store_contract<MAXQ>(P, j, b, acc, 2 * P.n_p, sh);
    ITEM_LOOP_END
}

// ------------------------------------------------------------------ even-odd Wilson, link-sharing groups
// rhs_block = 8 in even-odd mode: one CTA of 256 threads takes a block of 256
// consecutive half-field entries for eight slots of the work list, one warp
// per slot.  The block is processed 32 entries at a time: the CTA first
// stages the 32 sites' eight links in shared memory (lane index innermost, so
// that a warp reads consecutive words), then every warp applies the hops of
// its own slot at those 32 sites with the links from shared memory.  Each
// link crosses L2 once per eight right-hand sides instead of once per
// right-hand side (about 850 instead of 1400 bytes of L1/L2 traffic per site
// and right-hand side), and each warp reduces its own slot's dot products.
#define WEO_G 8                 // slots per work item (one warp each)
#define WEO_SUB 32              // entries per shared-memory link stage

#define ITEMG_LOOP(LIST)                                                        \
    const int cnt = P.counts[LIST];                                             \
    const int *lst = P.lists + (size_t)(LIST) * P.R;                            \
    const int ngrp_ = (cnt + WEO_G - 1) / WEO_G;                                \
    const int64_t n_items = (int64_t)ngrp_ * P.nsb;                             \
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;                  \
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {              \
        const int grp_ = (int)(it / P.nsb);                                     \
        const int b = (int)(it - (int64_t)grp_ * P.nsb);                        \
        const int jw = (grp_ * WEO_G + wid < cnt) ? lst[grp_ * WEO_G + wid] : -1; \
        const bool act = jw >= 0 && P.slots[jw].phase == PH_INNER;
#define ITEMG_LOOP_END }

// the eight links of the sites of entries base .. base + 31 (parity par) into
// sU[k][e][lane], k = 2 mu + (0 forward: U_mu(x), 1 backward: U_mu(x - mu))
template <typename R, typename LS>
__device__ __forceinline__ void weo_stage_links(const EP &P, int par, int base, Cx<R> (*sU)[9][WEO_SUB]) {
    // 32 sites x 8 links = 256 threads; warp k stages link k of the 32 sites,
    // consecutive entries of the even-odd ordered copy
    const int i = threadIdx.x & 31, k = threadIdx.x >> 5;
    const int h = base + i;
    if (h < P.nsite) {
        int x[4];
        const int s = half_site(P.g, par, h, x);
        const int mu = k >> 1;
        const int pos = (k & 1) ? eo_link_pos(P.g.N, nb_bwd(P.g, s, x, mu), 1 - par) : eo_link_pos(P.g.N, s, par);
        Cx<R> u[3][3];
        load_link<R, LS>((const LS *)P.U, P.g.N, mu, pos, u);
#pragma unroll
        for (int e = 0; e < 9; ++e) sU[k][e][i] = u[e / 3][e % 3];
    }
}

// (H psi)(x) at site idx (coordinates x) with the neighbour spinors read from
// the half field f (Nh entries) and the links from the staged sU column `col`
template <typename R, typename S>
__device__ __forceinline__ void wilson_hop_staged(const Geom &g, const S *f, int Nh, Cx<R> (*sU)[9][WEO_SUB],
                                                  int col, int antip, int idx, const int x[4], Cx<R> acc[4][3]) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[s][a] = Cx<R>{R(0), R(0)};
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        {   // forward hop: (1 - g_mu) U_mu(x) psi(x + mu)
            const int y = nb_fwd(g, idx, x, mu);
            const R eta = (antip && mu == 3 && x[3] == g.D[3] - 1) ? R(-1) : R(1);
            Cx<R> ps[4][3], h[2][3], uh[2][3];
            load_spinor<S, R>(f, Nh, y >> 1, ps);
            spin_project<R>(mu, R(-1), ps, h);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Cx<R> t = cmul(sU[2 * mu][3 * a][col], h[k][0]);
                    t = cadd(t, cmul(sU[2 * mu][3 * a + 1][col], h[k][1]));
                    t = cadd(t, cmul(sU[2 * mu][3 * a + 2][col], h[k][2]));
                    uh[k][a] = t;
                }
            spin_accumulate<R>(mu, R(-1), eta, uh, acc);
        }
        {   // backward hop: (1 + g_mu) U_mu(x - mu)^dagger psi(x - mu)
            const int y = nb_bwd(g, idx, x, mu);
            const R eta = (antip && mu == 3 && x[3] == 0) ? R(-1) : R(1);
            Cx<R> ps[4][3], h[2][3], uh[2][3];
            load_spinor<S, R>(f, Nh, y >> 1, ps);
            spin_project<R>(mu, R(1), ps, h);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Cx<R> t = cconjmul(sU[2 * mu + 1][a][col], h[k][0]);
                    t = cadd(t, cconjmul(sU[2 * mu + 1][3 + a][col], h[k][1]));
                    t = cadd(t, cconjmul(sU[2 * mu + 1][6 + a][col], h[k][2]));
                    uh[k][a] = t;
                }
            spin_accumulate<R>(mu, R(1), eta, uh, acc);
        }
    }
}

// grouped h = D_oe p (WHICH 0: p = pv; 1: p = s) at the odd entries
template <typename S, typename LS, int WHICH>
__global__ void __launch_bounds__(PT_BLOCK, std::is_same<S, double>::value ? 2 : PT_WIL_MINB) k_weo_hop_g(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ Cx<R> sU[8][9][WEO_SUB];
    const int N = P.nsite;
    ITEMG_LOOP(LIST_INNER)
        const S *src = act ? slot_cptr<S>(WHICH ? P.s : P.pv, jw, P.L) : nullptr;
        S *hf = act ? slot_ptr<S>(P.p1, jw, P.L) : nullptr;
        for (int sub = 0; sub < PT_BLOCK / WEO_SUB; ++sub) {
            const int base = b * PT_BLOCK + sub * WEO_SUB;
            if (base >= N) break;                              // uniform over the CTA
            __syncthreads();                                   // the previous stage is consumed
            weo_stage_links<R, LS>(P, 1, base, sU);
            __syncthreads();
            const int idx = base + lane;
            if (act && idx < N) {
                int xc[4];
                const int s = half_site(P.g, 1, idx, xc);
                Cx<R> acc[4][3], o[12];
                wilson_hop_staged<R, S>(P.g, src, N, sU, lane, P.antip, s, xc, acc);
#pragma unroll
                for (int c = 0; c < 12; ++c)
                    o[c] = Cx<R>{rnd<S, R>(acc[c / 3][c % 3].re), rnd<S, R>(acc[c / 3][c % 3].im)};
                store_spinor<S, R>(hf, N, idx, o);
            }
        }
    ITEMG_LOOP_END
}

// warp sums of K values, written by lane 0 as the partials of (slot jw, block b)
template <int K, typename R>
__device__ __forceinline__ void weo_warp_store(const EP &P, int jw, int b, R vr[K]) {
#pragma unroll
    for (int k = 0; k < K; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) vr[k] += __shfl_down_sync(0xffffffffu, vr[k], o);
    if ((threadIdx.x & 31) == 0) {
        double *dst = P.partials + ((size_t)jw * P.nsb + b) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) dst[k] = (double)vr[k];
    }
}

// grouped v = S p = p - kappa^2 D_eo h at the even entries;  partial (r0, v)
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BLOCK, std::is_same<S, double>::value ? 2 : PT_WIL_MINB) k_weo_apply1_g(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ Cx<R> sU[8][9][WEO_SUB];
    const int N = P.nsite;
    const R k2 = (R)(P.kappa * P.kappa);
    ITEMG_LOOP(LIST_INNER)
        const S *pv = act ? slot_cptr<S>(P.pv, jw, P.L) : nullptr;
        const S *h = act ? slot_cptr<S>(P.p1, jw, P.L) : nullptr;
        const S *r0 = act ? slot_cptr<S>(P.r0, jw, P.L) : nullptr;
        S *q = act ? slot_ptr<S>(P.q, jw, P.L) : nullptr;
        R vr[2] = {R(0), R(0)};
        for (int sub = 0; sub < PT_BLOCK / WEO_SUB; ++sub) {
            const int base = b * PT_BLOCK + sub * WEO_SUB;
            if (base >= N) break;
            __syncthreads();
            weo_stage_links<R, LS>(P, 0, base, sU);
            __syncthreads();
            const int idx = base + lane;
            if (act && idx < N) {
                int xc[4];
                const int s = half_site(P.g, 0, idx, xc);
                Cx<R> acc[4][3], ps[4][3], z[4][3], av[12];
                wilson_hop_staged<R, S>(P.g, h, N, sU, lane, P.antip, s, xc, acc);
                load_spinor<S, R>(pv, N, idx, ps);
                load_spinor<S, R>(r0, N, idx, z);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const Cx<R> w = csub(ps[c / 3][c % 3], cscale(acc[c / 3][c % 3], k2));
                    av[c] = Cx<R>{rnd<S, R>(w.re), rnd<S, R>(w.im)};
                    const Cx<R> zc = z[c / 3][c % 3];
                    vr[0] += zc.re * av[c].re + zc.im * av[c].im;
                    vr[1] += zc.re * av[c].im - zc.im * av[c].re;
                }
                store_spinor<S, R>(q, N, idx, av);
            }
        }
        if (act) weo_warp_store<2, R>(P, jw, b, vr);
    ITEMG_LOOP_END
}

// grouped t = S s = s - kappa^2 D_eo h at the even entries;  partials (t, s), |t|^2
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BLOCK, std::is_same<S, double>::value ? 2 : PT_WIL_MINB) k_weo_apply2_g(EP P) {
    typedef typename ArithT<S>::T R;
    __shared__ Cx<R> sU[8][9][WEO_SUB];
    const int N = P.nsite;
    const R k2 = (R)(P.kappa * P.kappa);
    ITEMG_LOOP(LIST_INNER)
        const S *sv = act ? slot_cptr<S>(P.s, jw, P.L) : nullptr;
        const S *h = act ? slot_cptr<S>(P.p1, jw, P.L) : nullptr;
        S *t = act ? slot_ptr<S>(P.t, jw, P.L) : nullptr;
        R vr[3] = {R(0), R(0), R(0)};
        for (int sub = 0; sub < PT_BLOCK / WEO_SUB; ++sub) {
            const int base = b * PT_BLOCK + sub * WEO_SUB;
            if (base >= N) break;
            __syncthreads();
            weo_stage_links<R, LS>(P, 0, base, sU);
            __syncthreads();
            const int idx = base + lane;
            if (act && idx < N) {
                int xc[4];
                const int s = half_site(P.g, 0, idx, xc);
                Cx<R> acc[4][3], sp[4][3], av[12];
                wilson_hop_staged<R, S>(P.g, h, N, sU, lane, P.antip, s, xc, acc);
                load_spinor<S, R>(sv, N, idx, sp);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const Cx<R> w = csub(sp[c / 3][c % 3], cscale(acc[c / 3][c % 3], k2));
                    av[c] = Cx<R>{rnd<S, R>(w.re), rnd<S, R>(w.im)};
                }
                store_spinor<S, R>(t, N, idx, av);
#pragma unroll
                for (int c = 0; c < 12; ++c) {
                    const Cx<R> tv = av[c], sc = sp[c / 3][c % 3];
                    vr[0] += tv.re * sc.re + tv.im * sc.im;
                    vr[1] += tv.re * sc.im - tv.im * sc.re;
                    vr[2] += tv.re * tv.re + tv.im * tv.im;
                }
            }
        }
        if (act) weo_warp_store<3, R>(P, jw, b, vr);
    ITEMG_LOOP_END
}

// ------------------------------------------------------------------ host driver
struct EngineRun {
    EP P;
    int grid_items;        // persistent CTAs of an item kernel without its own entry below
    int grid_warps;        // CTAs of the finalize kernels (8 warps each)
    int kernels_per_iter;
    // persistent grid of each item kernel: SMs x its own resident CTAs per SM
    int g_contract, g_oupd, g_ores, g_apply1, g_apply2, g_upd, g_s, g_dir;
    int g_apply1_x2, g_apply2_x2, g_contract32;
    int g_hop, g_ohop;                 // even-odd: the odd-site hop of the inner and of the outer step
    int g_obp;                         // even-odd Wilson: b'_e of new tasks
    int g_hop_g, g_apply1_g, g_apply2_g;   // even-odd Wilson, link-sharing groups of slots
    double *part_con, *part_outer;   // partial-sum regions of the contraction and outer kernel groups
};

template <typename K>
static int persistent_grid(K kernel, int num_sms, int block = PT_BLOCK) {
    int occ = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, block, 0) != cudaSuccess || occ < 1) {
        cudaGetLastError();
        occ = 1;
    }
    return num_sms * occ;
}

// Events recorded around kernel groups when profiling is on (9 per iteration):
// e0..e4 inner kernels, e5/e6 outer steps, e7/e8 whole iteration.
#define PT_EV_PER_ITER 9
static inline void ev_rec(const cudaEvent_t *ev, int i, cudaStream_t st) {
    if (ev) cudaEventRecordWithFlags(ev[i], st, cudaEventRecordExternal);
}

// One engine iteration.  With `side` (two capture side streams and three
// events; P.overlap set, so that the scheduler's three work lists are
// disjoint: a slot leaving the outer step starts its inner solve one
// iteration later) the contraction and the outer steps run as graph branches
// beside the inner kernels, each group on its own slots and its own
// partial-sum region: the FP64 residual (FP64-pipe bound) can share the GPU
// with the memory-bound inner kernels.  The branches join before the next
// iteration's scheduler.
template <int KIND, typename S, typename LS>
static void enqueue_iteration(const EngineRun &E, cudaStream_t st, const cudaEvent_t *ev, const cudaStream_t *side,
                              const cudaEvent_t *sev) {
    const EP &P = E.P;
    EP Pc = P, Po = P;               // the same parameters with the groups' own partial-sum regions
    Pc.partials = E.part_con;
    Po.partials = E.part_outer;
    const int W = E.grid_warps;
    ev_rec(ev, 7, st);
    k_schedule<<<1, 1024, 0, st>>>(P);
    cudaStream_t s_con = st, s_out = st;
    if (side) {
        cudaEventRecord(sev[0], st);
        cudaStreamWaitEvent(side[0], sev[0], 0);
        cudaStreamWaitEvent(side[1], sev[0], 0);
        s_con = side[0];
        s_out = side[1];
    }
    if (P.eo) {
        if constexpr (KIND == 0) {
            if (P.n_p <= 16) k_eo_contract<16><<<E.g_contract, P.bs, 0, s_con>>>(Pc);
            else k_eo_contract<PT_MAX_P><<<E.g_contract32, P.bs, 0, s_con>>>(Pc);
        } else {
            if (P.n_p <= 16) k_weo_contract<16><<<E.g_contract, P.bs, 0, s_con>>>(Pc);
            else k_weo_contract<PT_MAX_P><<<E.g_contract32, P.bs, 0, s_con>>>(Pc);
        }
    } else {
        if (P.n_p <= 16) k_contract<KIND, 16><<<E.g_contract, P.bs, 0, s_con>>>(Pc);
        else k_contract<KIND, PT_MAX_P><<<E.g_contract32, P.bs, 0, s_con>>>(Pc);
    }
    k_fin_contract<<<W, 256, 0, s_con>>>(Pc);
    ev_rec(ev, 5, s_out);
    k_outer_update<KIND, S><<<E.g_oupd, P.bs, 0, s_out>>>(Po);
    if (P.eo) {
        if constexpr (KIND == 0) {
            k_eo_outer_hop<<<E.g_ohop, P.bs, 0, s_out>>>(Po);
            k_eo_outer_residual<S><<<E.g_ores, P.bs, 0, s_out>>>(Po);
        } else {
            k_weo_outer_hop<<<E.g_ohop, P.bs, 0, s_out>>>(Po);
            k_weo_outer_bprime<<<E.g_obp, P.bs, 0, s_out>>>(Po);
            k_weo_outer_residual<S><<<E.g_ores, P.bs, 0, s_out>>>(Po);
        }
    } else {
        k_outer_residual<KIND, S><<<E.g_ores, P.bs, 0, s_out>>>(Po);
    }
    k_fin_outer<<<W, 256, 0, s_out>>>(Po);
    ev_rec(ev, 6, s_out);
    if constexpr (KIND == 0) {
        ev_rec(ev, 0, st);
        if (P.eo) {
            if (P.vec4) {
                k_eo_hop_v4<S><<<E.g_hop, P.bs, 0, st>>>(P);
                k_eo_apply_v4<S><<<E.g_apply1, P.bs, 0, st>>>(P);
            } else {
                k_eo_hop<S><<<E.g_hop, P.bs, 0, st>>>(P);
                k_eo_apply<S><<<E.g_apply1, P.bs, 0, st>>>(P);
            }
        } else if (P.vec4) {
            k_cg_apply_v4<S><<<E.g_apply1, P.bs, 0, st>>>(P);
        } else {
            k_cg_apply<S><<<E.g_apply1, P.bs, 0, st>>>(P);
        }
        ev_rec(ev, 1, st);
        k_fin_cg_alpha<<<W, 256, 0, st>>>(P);
        if (P.vec4) k_cg_update_v4<S><<<E.g_upd, P.bs, 0, st>>>(P);
        else k_cg_update<S><<<E.g_upd, P.bs, 0, st>>>(P);
        k_fin_cg_beta<<<W, 256, 0, st>>>(P);
        ev_rec(ev, 2, st);
    } else if (P.eo) {
        ev_rec(ev, 0, st);
        if (P.rhs_block == WEO_G) {
            k_weo_hop_g<S, LS, 0><<<E.g_hop_g, PT_BLOCK, 0, st>>>(P);
            k_weo_apply1_g<S, LS><<<E.g_apply1_g, PT_BLOCK, 0, st>>>(P);
        } else if (P.clover) {
            k_weo_hop<S, LS, 0, 1><<<E.g_hop, P.bs, 0, st>>>(P);
            k_weo_apply1<S, LS, 1><<<E.g_apply1, P.bs, 0, st>>>(P);
        } else {
            k_weo_hop<S, LS, 0><<<E.g_hop, P.bs, 0, st>>>(P);
            k_weo_apply1<S, LS><<<E.g_apply1, P.bs, 0, st>>>(P);
        }
        ev_rec(ev, 1, st);
        k_fin_bicg_alpha<<<W, 256, 0, st>>>(P);
        k_bicg_s<S><<<E.g_s, P.bs, 0, st>>>(P);
        ev_rec(ev, 2, st);
        if (P.rhs_block == WEO_G) {
            k_weo_hop_g<S, LS, 1><<<E.g_hop_g, PT_BLOCK, 0, st>>>(P);
            k_weo_apply2_g<S, LS><<<E.g_apply2_g, PT_BLOCK, 0, st>>>(P);
        } else if (P.clover) {
            k_weo_hop<S, LS, 1, 1><<<E.g_hop, P.bs, 0, st>>>(P);
            k_weo_apply2<S, LS, 1><<<E.g_apply2, P.bs, 0, st>>>(P);
        } else {
            k_weo_hop<S, LS, 1><<<E.g_hop, P.bs, 0, st>>>(P);
            k_weo_apply2<S, LS><<<E.g_apply2, P.bs, 0, st>>>(P);
        }
        ev_rec(ev, 3, st);
        k_fin_bicg_omega<<<W, 256, 0, st>>>(P);
        k_bicg_update<S><<<E.g_upd, P.bs, 0, st>>>(P);
        k_fin_bicg_beta<<<W, 256, 0, st>>>(P);
        k_bicg_dir<S><<<E.g_dir, P.bs, 0, st>>>(P);
        ev_rec(ev, 4, st);
    } else {
        ev_rec(ev, 0, st);
        if constexpr (!std::is_same<S, double>::value) {
            if (P.rhs_block == 2) k_bicg_apply1_x2<S, LS><<<E.g_apply1_x2, P.bs, 0, st>>>(P);
            else k_bicg_apply1<S, LS><<<E.g_apply1, P.bs, 0, st>>>(P);
        } else {
            k_bicg_apply1<S, LS><<<E.g_apply1, P.bs, 0, st>>>(P);
        }
        ev_rec(ev, 1, st);
        k_fin_bicg_alpha<<<W, 256, 0, st>>>(P);
        k_bicg_s<S><<<E.g_s, P.bs, 0, st>>>(P);
        ev_rec(ev, 2, st);
        if constexpr (!std::is_same<S, double>::value) {
            if (P.rhs_block == 2) k_bicg_apply2_x2<S, LS><<<E.g_apply2_x2, P.bs, 0, st>>>(P);
            else k_bicg_apply2<S, LS><<<E.g_apply2, P.bs, 0, st>>>(P);
        } else {
            k_bicg_apply2<S, LS><<<E.g_apply2, P.bs, 0, st>>>(P);
        }
        ev_rec(ev, 3, st);
        k_fin_bicg_omega<<<W, 256, 0, st>>>(P);
        k_bicg_update<S><<<E.g_upd, P.bs, 0, st>>>(P);
        k_fin_bicg_beta<<<W, 256, 0, st>>>(P);
        k_bicg_dir<S><<<E.g_dir, P.bs, 0, st>>>(P);
        ev_rec(ev, 4, st);
    }
    if (side) {
        cudaEventRecord(sev[1], side[0]);
        cudaEventRecord(sev[2], side[1]);
        cudaStreamWaitEvent(st, sev[1], 0);
        cudaStreamWaitEvent(st, sev[2], 0);
    }
    ev_rec(ev, 8, st);
}

// (class, start event, end event) of the timed kernel groups; class 0 = the
// operator apply of the inner Krylov iteration, 1 = inner vector updates,
// 2 = FP64 outer steps, 3 = whole engine iteration.
static const int PROF_PAIRS_LAP[4][3] = {{0, 0, 1}, {1, 1, 2}, {2, 5, 6}, {3, 7, 8}};
static const int PROF_PAIRS_WIL[6][3] = {{0, 0, 1}, {1, 1, 2}, {0, 2, 3}, {1, 3, 4}, {2, 5, 6}, {3, 7, 8}};

struct EngineRequest {
    int mode;
    int n_tasks;
    const Task *h_tasks;
    const int32_t *col;
    uint64_t seed;
    int noise, mu, n_p, dilute, pshift;
    const int *p_list;
    const double *B_user;
    double *X_user;
    double tol;
    int maxit;
    int prec;
    int R_force;               // >0: exact slot count (grad mode)
    int n_lev = 0, n_pr = 0, m_fin = 0;   // nested trace mode (see EP)
    const int32_t *lev_cols = nullptr;
    const int *lev_anc = nullptr;
    // outputs
    std::vector<double> task_out;   // trace: [n_tasks][n_p] complex
    std::vector<TaskStat> tstat;
    double *x64_out;           // grad mode: device pointer to the solutions (valid until next call)
    int R_used;
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// the even-odd split needs every side even (each hop then joins opposite parities)
static bool pt_evenodd_ok(const int dims[4]) {
    for (int mu = 0; mu < 4; ++mu)
        if (dims[mu] < 2 || dims[mu] % 2) return false;
    return true;
}

// Engine parameters for (operator kind, precision, lattice): the autotuner's
// candidate while it runs, else a stored tuning, else the defaults.
static pt_ctx::Tune engine_tuning(const pt_ctx *c, const pt_op *op, int prec) {
    if (c->in_trial) return c->trial;
    for (int i = 0; i < 16; ++i) {
        const pt_ctx::Tune &t = c->tune[i];
        if (t.used && t.kind == op->kind && t.prec == prec && !memcmp(t.dims, op->dims, sizeof(t.dims))) return t;
    }
    pt_ctx::Tune d;
    memset(&d, 0, sizeof(d));
    d.kind = op->kind;
    d.prec = prec;
    memcpy(d.dims, op->dims, sizeof(d.dims));
    d.delta = prec == PT_PREC_FP64 ? 0.0 : (prec == PT_PREC_MIXED_FP32 ? 1e-5 : 1e-2);
    d.group = op->kind ? 8 : 1;
    d.graph_iters = 8;
    d.rhs_block = 1;
    d.overlap = 0;
    d.evenodd = pt_evenodd_ok(op->dims) ? 1 : 0;
    d.cta_threads = 0;
    d.sites_per_thread = 0;
    return d;
}

template <int KIND, typename S, typename LS>
static int run_engine_t(const pt_op *op, EngineRequest &rq, pt_stats *stats) {
    pt_ctx *c = op->ctx;
    const Geom g = op->g;
    const pt_ctx::Tune tn = engine_tuning(c, op, rq.prec);
    // even-odd (every side even) unless switched off; the gradient works on
    // full-lattice solutions and keeps the full system
    const bool clv = KIND == 1 && op->csw != 0.0;
    const bool eo = (tn.evenodd || clv) && rq.mode != MODE_GRAD && pt_evenodd_ok(op->dims);
    if (clv && !eo) {
        pt_set_error("the clover operator runs on the even-odd engine only (every side even; no gradient)");
        return PT_ERR_ARG;
    }
    const int nsite = eo ? g.N / 2 : g.N;
    const int64_t L = eo ? (int64_t)nsite * (KIND ? 24 : 1) : pt_field_reals(op);
    // inner vectors: CG e, r, p (two buffers), q (+ t on the odd sites); BiCGStab
    // e, r, p, v, s, t, r0 (+ the odd-site hop buffer); FP64: x (+ t64, + b'_e)
    const int nvec = KIND ? (eo ? 8 : 7) : (eo ? 6 : 5);
    const int nf64 = eo ? 3 : 1;
    const size_t per_slot = (size_t)L * (nf64 * sizeof(double) + nvec * sizeof(S));
    // even-odd Wilson: the inner kernels read a copy of their links in the
    // even-odd order (LinkLayout<LS>::CHUNKS chunks per site)
    const size_t ueo_bytes = (KIND == 1 && eo) ? (size_t)g.N * LinkLayout<LS>::CHUNKS * sizeof(typename LinkLayout<LS>::E) : 0;
    const size_t budget = c->mem_budget > 2 * ueo_bytes ? c->mem_budget - ueo_bytes : c->mem_budget / 2;
    int R = rq.R_force > 0 ? rq.R_force : (int)std::min<size_t>((size_t)rq.n_tasks, budget / per_slot);
    if (rq.R_force <= 0 && c->max_slots > 0) R = std::min(R, c->max_slots);
    if (R < 1) R = 1;
    if (rq.R_force <= 0) R = std::min(R, 4096);
    // item geometry: CTA threads and sites per thread (the Laplacian's vector
    // path needs a multiple of 4 sites per thread)
    const int bs = tn.cta_threads ? tn.cta_threads : PT_BLOCK;
    const int spt = KIND ? 1 : (tn.sites_per_thread ? tn.sites_per_thread : Tile<0>::SPT);
    const int nsb = (int)(((int64_t)nsite + (int64_t)bs * spt - 1) / ((int64_t)bs * spt));
    const int K_MAX = 2 * PT_MAX_P;
    // layout of the work space
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    size_t o_x64 = take((size_t)R * L * sizeof(double));
    size_t o_t64 = eo ? take((size_t)R * L * sizeof(double)) : 0;
    size_t o_b64 = eo ? take((size_t)R * L * sizeof(double)) : 0;
    size_t o_vec[8];
    for (int v = 0; v < nvec; ++v) o_vec[v] = take((size_t)R * L * sizeof(S));
    size_t o_slots = take((size_t)R * sizeof(Slot));
    // partial sums per (slot, item): one region per kernel group (contraction, outer, inner), so that
    // the groups can run concurrently (their reductions use different strides)
    size_t o_part = take((size_t)R * nsb * K_MAX * sizeof(double));
    size_t o_part_outer = take((size_t)R * nsb * 4 * sizeof(double));
    size_t o_part_inner = take((size_t)R * nsb * 4 * sizeof(double));
    size_t o_cnt = take((size_t)R * sizeof(int));
    size_t o_lists = take((size_t)3 * R * sizeof(int));
    size_t o_counts = take(4 * sizeof(int));
    size_t o_head = take(sizeof(int));
    size_t o_flags = take(8 * sizeof(int));
    size_t o_tasks = take((size_t)rq.n_tasks * sizeof(Task));
    size_t o_tstat = take((size_t)rq.n_tasks * sizeof(TaskStat));
    size_t o_tout = take((size_t)rq.n_tasks * std::max(rq.n_p, 1) * 2 * sizeof(double));
    size_t o_ueo = ueo_bytes ? take(ueo_bytes) : 0;
    void *ws;
    int rc = pt_workspace(c, off, &ws);
    if (rc) return rc;
    char *base = (char *)ws;
    EngineRun E;
    EP &P = E.P;
    memset(&P, 0, sizeof(P));
    P.g = g;
    P.kind = KIND;
    P.nsb = nsb;
    P.bs = bs;
    P.spt = spt;
    P.R = R;
    P.eo = eo ? 1 : 0;
    P.nsite = nsite;
    P.gs = tn.group;
    // right-hand sides per Wilson work item: 2 on the full system (mixed
    // precision), a group of WEO_G slots (one warp each, links staged once in
    // shared memory) in even-odd mode with 256-thread CTAs
    P.rhs_block = 1;
    if (KIND == 1 && !eo && !std::is_same<S, double>::value && tn.rhs_block == 2) P.rhs_block = 2;
    if (KIND == 1 && eo && tn.rhs_block == WEO_G && bs == PT_BLOCK && !clv) P.rhs_block = WEO_G;
    P.overlap = tn.overlap ? 1 : 0;
    // four sites (even-odd: four half entries of one x row) per thread
    P.vec4 = (KIND == 0 && g.D[0] % (eo ? 8 : 4) == 0) ? 1 : 0;
    P.L = L;
    P.diag = 8.0 + op->m2;
    P.kappa = op->kappa;
    P.antip = op->antip;
    if constexpr (KIND == 1) {
        P.U = std::is_same<S, double>::value ? (const void *)op->U64
              : std::is_same<S, float>::value ? (const void *)op->U32 : (const void *)op->U16;
    }
    P.U64 = op->U64;
    P.clover = clv ? 1 : 0;
    P.CL32 = (const float4 *)op->CL32;
    P.CL64 = (const double2 *)op->CL64;
    P.mode = rq.mode;
    P.col = rq.col;
    P.seed = rq.seed;
    P.noise = rq.noise;
    P.mu = rq.mu;
    P.n_p = rq.n_p;
    P.n_lev = rq.n_lev;
    P.n_pr = rq.n_pr;
    P.m_fin = rq.m_fin;
    P.lev_cols = rq.lev_cols;
    P.lev_anc = rq.lev_anc;
    P.dilute = rq.dilute;
    P.pshift = rq.pshift;
    // displacements reduced to [0, D_mu) once here (the contractions add and
    // conditionally subtract instead of taking a modulo per site)
    for (int n = 0; n < rq.n_p && n < PT_MAX_P; ++n) {
        const int D = g.D[rq.mu];
        P.p[n] = ((rq.p_list[n] % D) + D) % D;
    }
    P.tasks = (const Task *)(base + o_tasks);
    P.n_tasks = rq.n_tasks;
    P.B_user = rq.B_user;
    P.X_user = rq.X_user;
    P.x64 = (double *)(base + o_x64);
    P.t64 = eo ? (double *)(base + o_t64) : nullptr;
    P.b64 = eo ? (double *)(base + o_b64) : nullptr;
    void **vp[8] = {&P.e, &P.r, &P.pv, &P.q, &P.s, &P.t, &P.r0, &P.p1};
    if constexpr (KIND == 0) vp[4] = &P.p1;     // CG: e, r, p (two buffers), q; even-odd adds t
    for (int v = 0; v < nvec; ++v) *vp[v] = base + o_vec[v];
    P.slots = (Slot *)(base + o_slots);
    P.partials = (double *)(base + o_part_inner);
    E.part_con = (double *)(base + o_part);
    E.part_outer = (double *)(base + o_part_outer);
    P.counters = (int *)(base + o_cnt);
    P.lists = (int *)(base + o_lists);
    P.counts = (int *)(base + o_counts);
    P.head = (int *)(base + o_head);
    P.flags = (int *)(base + o_flags);
    P.tstat = (TaskStat *)(base + o_tstat);
    P.task_out = (double *)(base + o_tout);
    P.tol = rq.tol;
    P.maxit = rq.maxit;
    P.delta = tn.delta;
    if (rq.prec == PT_PREC_FP64) P.max_inner = rq.maxit;
    else if (rq.prec == PT_PREC_MIXED_FP32) P.max_inner = 4000;
    else P.max_inner = 400;

    cudaStream_t st = c->stream;
    PT_CUDA(cudaMemcpyAsync((void *)P.tasks, rq.h_tasks, (size_t)rq.n_tasks * sizeof(Task), cudaMemcpyHostToDevice, st));
    PT_CUDA(cudaMemsetAsync(P.slots, 0, (size_t)R * sizeof(Slot), st));   // phase EMPTY
    PT_CUDA(cudaMemsetAsync(P.counters, 0, (size_t)R * sizeof(int), st));
    PT_CUDA(cudaMemsetAsync(P.head, 0, sizeof(int), st));
    PT_CUDA(cudaMemsetAsync(P.flags, 0, 8 * sizeof(int), st));
    PT_CUDA(cudaMemsetAsync(P.tstat, 0, (size_t)rq.n_tasks * sizeof(TaskStat), st));
    PT_CUDA(cudaMemsetAsync(P.task_out, 0, (size_t)rq.n_tasks * std::max(rq.n_p, 1) * 2 * sizeof(double), st));
    // zero the vectors once so that no slot ever reads uninitialised memory
    PT_CUDA(cudaMemsetAsync(base + o_x64, 0, o_slots - o_x64, st));
    if constexpr (KIND == 1) {
        if (ueo_bytes) {
            typedef typename LinkLayout<LS>::E E;
            E *ueo = (E *)(base + o_ueo);
            k_links_eo<E><<<c->num_sms * 8, 256, 0, st>>>(g, LinkLayout<LS>::CHUNKS, (const E *)P.U, ueo);
            PT_CUDA(cudaGetLastError());
            P.U = ueo;
        }
    }

    int occ = 0;
    if constexpr (KIND == 0) {
        PT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_apply<S>, bs, 0));
    } else {
        PT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bicg_apply1<S, LS>, bs, 0));
    }
    occ = std::max(occ, 1);
    E.grid_items = c->num_sms * occ;
    const int ns = c->num_sms;
    E.g_contract = persistent_grid(k_contract<KIND, 16>, ns, bs);
    E.g_contract32 = persistent_grid(k_contract<KIND, PT_MAX_P>, ns, bs);
    E.g_oupd = persistent_grid(k_outer_update<KIND, S>, ns, bs);
    E.g_ores = persistent_grid(k_outer_residual<KIND, S>, ns, bs);
    E.g_hop = E.g_ohop = E.g_obp = 0;
    E.g_hop_g = E.g_apply1_g = E.g_apply2_g = 0;
    if constexpr (KIND == 0) {
        if (eo) {
            E.g_contract = persistent_grid(k_eo_contract<16>, ns, bs);
            E.g_contract32 = persistent_grid(k_eo_contract<PT_MAX_P>, ns, bs);
            E.g_ores = persistent_grid(k_eo_outer_residual<S>, ns, bs);
            E.g_ohop = persistent_grid(k_eo_outer_hop, ns, bs);
            E.g_apply1 = E.g_apply2 = P.vec4 ? persistent_grid(k_eo_apply_v4<S>, ns, bs)
                                             : persistent_grid(k_eo_apply<S>, ns, bs);
            E.g_hop = P.vec4 ? persistent_grid(k_eo_hop_v4<S>, ns, bs) : persistent_grid(k_eo_hop<S>, ns, bs);
        } else {
            E.g_apply1 = E.g_apply2 = P.vec4 ? persistent_grid(k_cg_apply_v4<S>, ns, bs)
                                             : persistent_grid(k_cg_apply<S>, ns, bs);
        }
        E.g_upd = P.vec4 ? persistent_grid(k_cg_update_v4<S>, ns, bs) : persistent_grid(k_cg_update<S>, ns, bs);
        E.g_s = E.g_dir = E.g_upd;
    } else if (eo) {
        E.g_contract = persistent_grid(k_weo_contract<16>, ns, bs);
        E.g_contract32 = persistent_grid(k_weo_contract<PT_MAX_P>, ns, bs);
        E.g_ores = persistent_grid(k_weo_outer_residual<S>, ns, bs);
        E.g_ohop = persistent_grid(k_weo_outer_hop, ns, bs);
        E.g_obp = persistent_grid(k_weo_outer_bprime, ns, bs);
        E.g_hop = clv ? persistent_grid(k_weo_hop<S, LS, 0, 1>, ns, bs) : persistent_grid(k_weo_hop<S, LS, 0>, ns, bs);
        E.g_apply1 = clv ? persistent_grid(k_weo_apply1<S, LS, 1>, ns, bs)
                         : persistent_grid(k_weo_apply1<S, LS>, ns, bs);
        E.g_apply2 = clv ? persistent_grid(k_weo_apply2<S, LS, 1>, ns, bs)
                         : persistent_grid(k_weo_apply2<S, LS>, ns, bs);
        E.g_apply1_x2 = E.g_apply2_x2 = 0;
        E.g_hop_g = persistent_grid(k_weo_hop_g<S, LS, 0>, ns, PT_BLOCK);
        E.g_apply1_g = persistent_grid(k_weo_apply1_g<S, LS>, ns, PT_BLOCK);
        E.g_apply2_g = persistent_grid(k_weo_apply2_g<S, LS>, ns, PT_BLOCK);
        E.g_upd = persistent_grid(k_bicg_update<S>, ns, bs);
        E.g_s = persistent_grid(k_bicg_s<S>, ns, bs);
        E.g_dir = persistent_grid(k_bicg_dir<S>, ns, bs);
    } else {
        E.g_apply1 = persistent_grid(k_bicg_apply1<S, LS>, ns, bs);
        E.g_apply2 = persistent_grid(k_bicg_apply2<S, LS>, ns, bs);
        if constexpr (!std::is_same<S, double>::value) {
            E.g_apply1_x2 = persistent_grid(k_bicg_apply1_x2<S, LS>, ns, bs);
            E.g_apply2_x2 = persistent_grid(k_bicg_apply2_x2<S, LS>, ns, bs);
        } else {
            E.g_apply1_x2 = E.g_apply2_x2 = 0;
        }
        E.g_upd = persistent_grid(k_bicg_update<S>, ns, bs);
        E.g_s = persistent_grid(k_bicg_s<S>, ns, bs);
        E.g_dir = persistent_grid(k_bicg_dir<S>, ns, bs);
    }
    E.grid_warps = std::max(1, std::min((R + 7) / 8, c->num_sms * 4));
    E.kernels_per_iter = KIND ? (eo ? 18 : 14) : (eo ? 12 : 10);

    // capture ITERS engine iterations into one graph
    const int ITERS = tn.graph_iters;
    std::vector<cudaEvent_t> evs;
    if (c->prof) {
        evs.resize(ITERS * PT_EV_PER_ITER);
        for (auto &e : evs) PT_CUDA(cudaEventCreate(&e));
    }
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    PT_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < ITERS; ++i)
        enqueue_iteration<KIND, S, LS>(E, c->cap_stream, c->prof ? &evs[(size_t)i * PT_EV_PER_ITER] : nullptr,
                                       tn.overlap ? c->cap_side : nullptr, c->cap_ev);
    cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
    if (ce != cudaSuccess) return pt_cuda_fail(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) { cudaGraphDestroy(graph); return pt_cuda_fail(ce, "cudaGraphInstantiate", __FILE__, __LINE__); }

    // bounded host loop: every RHS stops within maxit Krylov iterations, plus a
    // few engine iterations per outer restart and per retire/refill
    const int64_t waves = (rq.n_tasks + R - 1) / R + 1;
    int64_t max_launches = waves * ((int64_t)rq.maxit * 2 + 400) / ITERS + 64;
    if (c->launch_limit > 0) max_launches = std::min(max_launches, c->launch_limit);
    int64_t launches = 0;
    int rc_loop = PT_OK;
    int *hf = c->h_flags;
    const int (*pairs)[3] = KIND ? PROF_PAIRS_WIL : PROF_PAIRS_LAP;
    const int n_pairs = KIND ? 6 : 4;
    while (true) {
        ce = cudaGraphLaunch(exec, c->stream);
        if (ce != cudaSuccess) { rc_loop = pt_cuda_fail(ce, "cudaGraphLaunch", __FILE__, __LINE__); break; }
        ++launches;
        ce = cudaMemcpyAsync(hf, P.flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
        if (ce != cudaSuccess) { rc_loop = pt_cuda_fail(ce, "engine flag read", __FILE__, __LINE__); break; }
        if (c->prof) {
            for (int i = 0; i < ITERS; ++i)
                for (int q = 0; q < n_pairs; ++q) {
                    float ms = 0.f;
                    const cudaEvent_t *ev = &evs[(size_t)i * PT_EV_PER_ITER];
                    if (cudaEventElapsedTime(&ms, ev[pairs[q][1]], ev[pairs[q][2]]) == cudaSuccess) {
                        c->prof_ms[pairs[q][0]] += ms;
                        c->prof_launches[pairs[q][0]] += 1;
                    }
                }
        }
        if (hf[FLAG_DONE]) break;
        if (launches >= max_launches) {
            pt_set_error("solver engine did not finish within %lld graph launches", (long long)max_launches);
            rc_loop = PT_ERR_TIMEOUT;
            break;
        }
    }
    for (auto &e : evs) cudaEventDestroy(e);
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    pt_kernel_launch_count += launches * ITERS * E.kernels_per_iter;
    int flag_numeric = hf[FLAG_NUMERIC], n_noconv = hf[FLAG_NOCONV];
    if (rc_loop) return rc_loop;

    rq.tstat.resize(rq.n_tasks);
    PT_CUDA(cudaMemcpyAsync(rq.tstat.data(), P.tstat, (size_t)rq.n_tasks * sizeof(TaskStat), cudaMemcpyDeviceToHost, st));
    if (rq.mode == MODE_TRACE) {
        rq.task_out.resize((size_t)rq.n_tasks * rq.n_p * 2);
        PT_CUDA(cudaMemcpyAsync(rq.task_out.data(), P.task_out, rq.task_out.size() * sizeof(double),
                                cudaMemcpyDeviceToHost, st));
    }
    PT_CUDA(cudaStreamSynchronize(st));
    rq.x64_out = P.x64;
    rq.R_used = R;
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->n_rhs = rq.n_tasks;
        stats->n_slots = R;
        stats->engine_iters = launches * ITERS;
        stats->graph_launches = launches;
        stats->kernel_launches = launches * ITERS * E.kernels_per_iter;
        for (auto &t : rq.tstat) {
            stats->inner_iters += t.iters;
            stats->outer_iters += t.outer;
            stats->max_relres = std::max(stats->max_relres, t.relres);
        }
        const int applies_per_it = KIND ? 2 : 1;
        // outer iterations after the first each apply A once in FP64
        stats->site_rhs_applies =
            (stats->inner_iters * applies_per_it + stats->outer_iters - stats->n_rhs) * (int64_t)g.N;
        stats->n_noconv = n_noconv;
    }
    if (flag_numeric & 1) {
        pt_set_error("non-finite residual (NaN/Inf) in the solve");
        return PT_ERR_NUMERIC;
    }
    if (n_noconv) {
        pt_set_error("%d right-hand side(s) did not reach tol %.3g within maxit %d", n_noconv, rq.tol, rq.maxit);
        return PT_ERR_NOCONV;
    }
    return PT_OK;
}

static int run_engine(const pt_op *op, EngineRequest &rq, pt_stats *stats) {
    if (op->kind == 0) {
        switch (rq.prec) {
            case PT_PREC_FP64: return run_engine_t<0, double, double>(op, rq, stats);
            case PT_PREC_MIXED_FP32: return run_engine_t<0, float, float>(op, rq, stats);
            case PT_PREC_MIXED_BF16: return run_engine_t<0, __nv_bfloat16, __nv_bfloat16>(op, rq, stats);
        }
    } else {
        switch (rq.prec) {
            case PT_PREC_FP64: return run_engine_t<1, double, double>(op, rq, stats);
            case PT_PREC_MIXED_FP32: return run_engine_t<1, float, float>(op, rq, stats);
            case PT_PREC_MIXED_BF16: return run_engine_t<1, __nv_bfloat16, __nv_bfloat16>(op, rq, stats);
        }
    }
    pt_set_error("unknown precision mode %d", rq.prec);
    return PT_ERR_ARG;
}

static int check_solver_args(int prec, double tol, int maxit) {
    PT_CHECK_ARG(prec == PT_PREC_FP64 || prec == PT_PREC_MIXED_FP32 || prec == PT_PREC_MIXED_BF16,
                 "unknown precision mode %d", prec);
    PT_CHECK_ARG(tol > 0.0 && tol < 1.0, "tol must be in (0, 1)");
    PT_CHECK_ARG(maxit >= 1 && maxit <= 10000000, "maxit must be in [1, 1e7]");
    return PT_OK;
}

// ------------------------------------------------------------------ pt_solve
extern "C" int pt_solve(pt_ctx *c, const pt_op *op, const double *B_dev, double *X_dev, int nrhs, int prec,
                        double tol, int maxit, int *iters_out, double *relres_out, pt_stats *stats) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_solve: bad context/operator");
    PT_CHECK_ARG(nrhs >= 0, "pt_solve: nrhs < 0");
    int rc = check_solver_args(prec, tol, maxit);
    if (rc) return rc;
    if (nrhs == 0) { if (stats) memset(stats, 0, sizeof(*stats)); return PT_OK; }
    PT_CHECK_ARG(B_dev && X_dev, "pt_solve: NULL field");
    PT_CUDA(cudaSetDevice(c->device));
    std::vector<Task> tasks(nrhs);
    for (int i = 0; i < nrhs; ++i) tasks[i] = Task{i, 0, 0, 0, 0, 0, 0, 0};
    EngineRequest rq;
    rq.mode = MODE_SOLVE;
    rq.n_tasks = nrhs;
    rq.h_tasks = tasks.data();
    rq.col = nullptr;
    rq.seed = 0;
    rq.noise = 0; rq.mu = 0; rq.n_p = 0; rq.dilute = 1; rq.pshift = 0;
    rq.p_list = nullptr;
    rq.B_user = B_dev;
    rq.X_user = X_dev;
    rq.tol = tol;
    rq.maxit = maxit;
    rq.prec = prec;
    rq.R_force = 0;
    rc = run_engine(op, rq, stats);
    if (rc == PT_OK || rc == PT_ERR_NOCONV) {
        for (int i = 0; i < nrhs && (int)rq.tstat.size() == nrhs; ++i) {
            if (iters_out) iters_out[i] = rq.tstat[i].iters;
            if (relres_out) relres_out[i] = rq.tstat[i].relres;
        }
    }
    return rc;
}

// ------------------------------------------------------------------ pt_trace_PAinv
static void build_probe_tasks(int cidx, int n_colours, int set0, int n_sets, int dof, int dilute, int adj_pairs,
                              std::vector<Task> &tasks) {
    const int ncomp = dilute ? dof : 1;
    for (int s = 0; s < n_sets; ++s)
        for (int col = 0; col < n_colours; ++col)
            for (int a = 0; a < ncomp; ++a) {
                tasks.push_back(Task{set0 + s, col, dilute ? a : -1, 0, cidx, 0, 0, 0});
                if (adj_pairs) tasks.push_back(Task{set0 + s, col, dilute ? a : -1, TASK_ADJ, cidx, 0, 0, 0});
            }
}

extern "C" int pt_trace_PAinv_multi(pt_ctx *c, const pt_op *op, int n_col, const int32_t *cols_dev,
                                    const int *n_colours, int mu, const int *p_list, int n_p, int noise, uint64_t seed,
                                    int set0, int n_sets, int dilute, int prec, double tol, int maxit, double *est_out,
                                    pt_stats *stats) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_trace_PAinv: bad context/operator");
    PT_CHECK_ARG(cols_dev && est_out && n_colours && n_col >= 1, "pt_trace_PAinv: NULL colour or output array");
    PT_CHECK_ARG(n_sets >= 1 && set0 >= 0, "pt_trace_PAinv: need n_sets >= 1, set0 >= 0");
    for (int i = 0; i < n_col; ++i)
        PT_CHECK_ARG(n_colours[i] >= 1 && n_colours[i] <= op->g.N, "pt_trace_PAinv: n_colours out of range");
    PT_CHECK_ARG(mu >= 0 && mu < 4, "pt_trace_PAinv: mu must be in 0..3");
    PT_CHECK_ARG(n_p >= 1 && n_p <= PT_MAX_P && p_list, "pt_trace_PAinv: 1 <= n_p <= %d", PT_MAX_P);
    PT_CHECK_ARG(noise == PT_NOISE_Z2 || (noise == PT_NOISE_Z4 && op->dof == 12),
                 "pt_trace_PAinv: Z4 noise needs the complex (Wilson) operator");
    int rc = check_solver_args(prec, tol, maxit);
    if (rc) return rc;
    int64_t n_tasks = 0;
    for (int i = 0; i < n_col; ++i) n_tasks += (int64_t)n_colours[i] * n_sets * (dilute ? op->dof : 1);
    PT_CHECK_ARG(n_tasks < (1LL << 30), "pt_trace_PAinv: too many right-hand sides");
    PT_CUDA(cudaSetDevice(c->device));
    std::vector<Task> tasks;
    tasks.reserve((size_t)n_tasks);
    for (int i = 0; i < n_col; ++i) build_probe_tasks(i, n_colours[i], set0, n_sets, op->dof, dilute, 0, tasks);
    EngineRequest rq;
    rq.mode = MODE_TRACE;
    rq.n_tasks = (int)tasks.size();
    rq.h_tasks = tasks.data();
    rq.col = cols_dev;
    rq.seed = seed;
    rq.noise = noise; rq.mu = mu; rq.n_p = n_p; rq.dilute = dilute ? 1 : 0; rq.pshift = 0;
    rq.p_list = p_list;
    rq.B_user = nullptr;
    rq.X_user = nullptr;
    rq.tol = tol;
    rq.maxit = maxit;
    rq.prec = prec;
    rq.R_force = 0;
    rc = run_engine(op, rq, stats);
    if (rc != PT_OK && rc != PT_ERR_NOCONV) return rc;
    // per (colouring, set) sums in the fixed task order (deterministic)
    for (size_t i = 0; i < (size_t)n_col * n_sets * n_p * 2; ++i) est_out[i] = 0.0;
    for (size_t t = 0; t < tasks.size(); ++t) {
        const size_t row = ((size_t)tasks[t].cidx * n_sets + (tasks[t].set - set0)) * n_p;
        for (int n = 0; n < n_p; ++n) {
            est_out[(row + n) * 2] += rq.task_out[(t * n_p + n) * 2];
            est_out[(row + n) * 2 + 1] += rq.task_out[(t * n_p + n) * 2 + 1];
        }
    }
    return rc;
}

extern "C" int pt_trace_PAinv(pt_ctx *c, const pt_op *op, const int32_t *col_dev, int n_colours, int mu,
                              const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets, int dilute,
                              int prec, double tol, int maxit, double *est_out, double *mean_out, double *var_out,
                              pt_stats *stats) {
    int rc = pt_trace_PAinv_multi(c, op, 1, col_dev, &n_colours, mu, p_list, n_p, noise, seed, set0, n_sets, dilute,
                                  prec, tol, maxit, est_out, stats);
    if (rc != PT_OK && rc != PT_ERR_NOCONV) return rc;
    for (int n = 0; n < n_p; ++n) {
        double mr = 0.0, mi = 0.0;
        for (int s = 0; s < n_sets; ++s) { mr += est_out[(s * n_p + n) * 2]; mi += est_out[(s * n_p + n) * 2 + 1]; }
        mr /= n_sets; mi /= n_sets;
        if (mean_out) { mean_out[2 * n] = mr; mean_out[2 * n + 1] = mi; }
        if (var_out) {
            double v = 0.0;
            for (int s = 0; s < n_sets; ++s) {
                double dr = est_out[(s * n_p + n) * 2] - mr, di = est_out[(s * n_p + n) * 2 + 1] - mi;
                v += dr * dr + di * di;
            }
            var_out[n] = n_sets > 1 ? v / (n_sets - 1) : 0.0;
        }
    }
    return rc;
}

// ------------------------------------------------------------------ nested trace
// Ancestor table anc[l][c] = level-l colour of the nodes of finest class c, and
// a flag when some node's level-l colour differs from it (not nested) or a
// finest colour is out of range.
__global__ void k_nest_anc(int N, int n_lev, int m_fin, const int32_t *__restrict__ cols, int *anc, int *bad) {
    const int32_t *fin = cols + (size_t)(n_lev - 1) * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const int c = fin[x];
        if (c < 0 || c >= m_fin) { atomicOr(bad, 1); continue; }
        for (int l = 0; l < n_lev; ++l) anc[(size_t)l * m_fin + c] = cols[(size_t)l * N + x];
    }
}

__global__ void k_nest_check(int N, int n_lev, int m_fin, const int32_t *__restrict__ cols,
                             const int *__restrict__ anc, int *bad) {
    const int32_t *fin = cols + (size_t)(n_lev - 1) * N;
    for (int x = blockIdx.x * blockDim.x + threadIdx.x; x < N; x += gridDim.x * blockDim.x) {
        const int c = fin[x];
        if (c < 0 || c >= m_fin) continue;
        for (int l = 0; l < n_lev; ++l)
            if (cols[(size_t)l * N + x] != anc[(size_t)l * m_fin + c]) atomicOr(bad, 2);
    }
}

extern "C" int pt_trace_PAinv_nested(pt_ctx *c, const pt_op *op, int n_lev, const int32_t *cols_dev,
                                     const int *n_colours, int mu, const int *p_list, int n_p, int noise,
                                     uint64_t seed, int set0, int n_sets, int dilute, int prec, double tol, int maxit,
                                     double *est_out, pt_stats *stats) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_trace_PAinv_nested: bad context/operator");
    PT_CHECK_ARG(cols_dev && est_out && n_colours && p_list && n_lev >= 1, "pt_trace_PAinv_nested: NULL argument");
    PT_CHECK_ARG(n_p >= 1 && n_lev * n_p <= PT_MAX_P, "pt_trace_PAinv_nested: need n_lev * n_p <= %d", PT_MAX_P);
    PT_CHECK_ARG(n_sets >= 1 && set0 >= 0 && mu >= 0 && mu < 4, "pt_trace_PAinv_nested: bad sets or mu");
    PT_CHECK_ARG(noise == PT_NOISE_Z2 || (noise == PT_NOISE_Z4 && op->dof == 12),
                 "pt_trace_PAinv_nested: Z4 noise needs the complex (Wilson) operator");
    const int m_fin = n_colours[n_lev - 1];
    PT_CHECK_ARG(m_fin >= 1 && m_fin <= op->g.N, "pt_trace_PAinv_nested: n_colours out of range");
    int rc = check_solver_args(prec, tol, maxit);
    if (rc) return rc;
    PT_CUDA(cudaSetDevice(c->device));
    const int N = op->g.N;
    int *anc = nullptr;
    PT_CUDA(cudaMallocAsync((void **)&anc, ((size_t)n_lev * m_fin + 64) * sizeof(int), c->stream));
    int *bad = anc + (size_t)n_lev * m_fin;
    PT_CUDA(cudaMemsetAsync(anc, 0xff, ((size_t)n_lev * m_fin + 64) * sizeof(int), c->stream));
    PT_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), c->stream));
    const int blocks = (int)std::min<long>(((long)N + 255) / 256, 16L * c->num_sms);
    k_nest_anc<<<blocks, 256, 0, c->stream>>>(N, n_lev, m_fin, cols_dev, anc, bad);
    k_nest_check<<<blocks, 256, 0, c->stream>>>(N, n_lev, m_fin, cols_dev, anc, bad);
    pt_kernel_launch_count += 2;
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaMemcpyAsync(c->h_flags, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaStreamSynchronize(c->stream));
    if (c->h_flags[0]) {
        const int f = c->h_flags[0];
        cudaFreeAsync(anc, c->stream);
        PT_CHECK_ARG(false, "pt_trace_PAinv_nested: %s", (f & 1) ? "finest colours outside [0, n_colours)"
                                                                   : "colourings are not nested");
    }
    std::vector<Task> tasks;
    build_probe_tasks(0, m_fin, set0, n_sets, op->dof, dilute, 0, tasks);
    std::vector<int> p_ext((size_t)n_lev * n_p);
    for (int q = 0; q < n_lev * n_p; ++q) p_ext[q] = p_list[q % n_p];
    EngineRequest rq;
    rq.mode = MODE_TRACE;
    rq.n_tasks = (int)tasks.size();
    rq.h_tasks = tasks.data();
    rq.col = cols_dev + (size_t)(n_lev - 1) * N;
    rq.seed = seed;
    rq.noise = noise; rq.mu = mu; rq.n_p = n_lev * n_p; rq.dilute = dilute ? 1 : 0; rq.pshift = 0;
    rq.p_list = p_ext.data();
    rq.B_user = nullptr;
    rq.X_user = nullptr;
    rq.tol = tol;
    rq.maxit = maxit;
    rq.prec = prec;
    rq.R_force = 0;
    rq.n_lev = n_lev;
    rq.n_pr = n_p;
    rq.m_fin = m_fin;
    rq.lev_cols = cols_dev;
    rq.lev_anc = anc;
    rc = run_engine(op, rq, stats);
    cudaFreeAsync(anc, c->stream);
    if (rc != PT_OK && rc != PT_ERR_NOCONV) return rc;
    // est[l][s][n] = sum over the finest classes of their contraction with the level-l probe
    const int Q = n_lev * n_p;
    for (size_t i = 0; i < (size_t)n_lev * n_sets * n_p * 2; ++i) est_out[i] = 0.0;
    for (size_t t = 0; t < tasks.size(); ++t)
        for (int q = 0; q < Q; ++q) {
            const int l = q / n_p, n = q % n_p;
            const size_t o = (((size_t)l * n_sets + (tasks[t].set - set0)) * n_p + n) * 2;
            est_out[o] += rq.task_out[(t * Q + q) * 2];
            est_out[o + 1] += rq.task_out[(t * Q + q) * 2 + 1];
        }
    return rc;
}

// ------------------------------------------------------------------ pt_grad
// per probe pair (slot 2i = x, slot 2i+1 = w, y = g5 w for Wilson, y = w for the
// Laplacian): dots y^H x and y^H v, and for Wilson the link outer products.
template <int KIND>
__global__ void k_grad_dots(EP P, int n_pairs, double *out /* [n_pairs][4] */) {
    __shared__ double sh[32 * 4];
    const int N = P.g.N;
    for (int64_t it = blockIdx.x; it < (int64_t)n_pairs * P.nsb; it += gridDim.x) {
        const int b = (int)(it % P.nsb), i = (int)(it / P.nsb);
        const int idx = b * PT_BS + threadIdx.x;
        double v[4] = {0.0, 0.0, 0.0, 0.0};
        const Task tk = P.tasks[2 * i];
        if (idx < N) {
            int xc[4];
            site_coords(P.g, idx, xc);
            const double *x = P.x64 + (size_t)(2 * i) * P.L;
            const double *w = P.x64 + (size_t)(2 * i + 1) * P.L;
            const uint64_t key = pt_set_key(P.seed, tk.set);
            const int NC = KIND ? 12 : 1;
            for (int cc = 0; cc < NC; ++cc) {
                Cx<double> y = Fld<KIND, double>::ld(w, N, cc, idx);
                if (KIND && cc >= 6) y = Cx<double>{-y.re, -y.im};
                Cx<double> xv = Fld<KIND, double>::ld(x, N, cc, idx);
                Cx<double> vv = source_val<KIND>(P, tk, key, idx, xc, cc);
                Cx<double> a1 = cconjmul(y, xv), a2 = cconjmul(y, vv);
                v[0] += a1.re; v[1] += a1.im; v[2] += a2.re; v[3] += a2.im;
            }
        }
        block_sum<4>(v, sh);
        if (threadIdx.x == 0)
            for (int k = 0; k < 4; ++k) out[((size_t)i * P.nsb + b) * 4 + k] = v[k];
        __syncthreads();
    }
}

// G_mu(x)_ab += kappa eta sum_{s} conj(y(x)_{s,a}) [(1 - g_mu) x(x+mu)]_{s,b}
// Gbar_mu(x)_ab += kappa eta sum_{s} conj(y(x+mu)_{s,b}) [(1 + g_mu) x(x)]_{s,a}
__global__ void k_grad_links(EP P, int n_pairs, double *G, double *Gb) {
    const int N = P.g.N;
    int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (gid >= (int64_t)N * 4) return;
    const int idx = (int)(gid >> 2), mu = (int)(gid & 3);
    int xc[4];
    site_coords(P.g, idx, xc);
    const int f = nb_fwd(P.g, idx, xc, mu);
    const double eta = (P.antip && mu == 3 && xc[3] == P.g.D[3] - 1) ? -1.0 : 1.0;
    Cx<double> g[3][3], gb[3][3];
    for (int a = 0; a < 3; ++a)
        for (int bb = 0; bb < 3; ++bb) { g[a][bb] = Cx<double>{0.0, 0.0}; gb[a][bb] = Cx<double>{0.0, 0.0}; }
    for (int i = 0; i < n_pairs; ++i) {
        const double *x = P.x64 + (size_t)(2 * i) * P.L;
        const double *w = P.x64 + (size_t)(2 * i + 1) * P.L;
        Cx<double> ps[4][3], h[2][3], wv[4][3];
        // (1 - g_mu) x(x + mu)
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a) { ps[s][a] = ld_cx<double, double>(x, N, 3 * s + a, f); wv[s][a] = Cx<double>{0, 0}; }
        spin_project<double>(mu, -1.0, ps, h);
        spin_accumulate<double>(mu, -1.0, 1.0, h, wv);
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a) {
                Cx<double> y = ld_cx<double, double>(w, N, 3 * s + a, idx);
                if (s >= 2) y = Cx<double>{-y.re, -y.im};
                for (int bb = 0; bb < 3; ++bb) g[a][bb] = cadd(g[a][bb], cconjmul(y, wv[s][bb]));
            }
        // (1 + g_mu) x(x)
        for (int s = 0; s < 4; ++s)
            for (int a = 0; a < 3; ++a) { ps[s][a] = ld_cx<double, double>(x, N, 3 * s + a, idx); wv[s][a] = Cx<double>{0, 0}; }
        spin_project<double>(mu, 1.0, ps, h);
        spin_accumulate<double>(mu, 1.0, 1.0, h, wv);
        for (int s = 0; s < 4; ++s)
            for (int bb = 0; bb < 3; ++bb) {
                Cx<double> y = ld_cx<double, double>(w, N, 3 * s + bb, f);
                if (s >= 2) y = Cx<double>{-y.re, -y.im};
                for (int a = 0; a < 3; ++a) gb[a][bb] = cadd(gb[a][bb], cconjmul(y, wv[s][a]));
            }
    }
    const double kw = P.kappa * eta;
    double *go = G + ((size_t)idx * 4 + mu) * 18;
    double *gbo = Gb + ((size_t)idx * 4 + mu) * 18;
    for (int a = 0; a < 3; ++a)
        for (int bb = 0; bb < 3; ++bb) {
            go[(a * 3 + bb) * 2] += kw * g[a][bb].re;
            go[(a * 3 + bb) * 2 + 1] += kw * g[a][bb].im;
            gbo[(a * 3 + bb) * 2] += kw * gb[a][bb].re;
            gbo[(a * 3 + bb) * 2 + 1] += kw * gb[a][bb].im;
        }
}

extern "C" int pt_grad(pt_ctx *c, const pt_op *op, const int32_t *col_dev, int n_colours, int mu, int p, int noise,
                       uint64_t seed, int set0, int n_sets, int dilute, int prec, double tol, int maxit,
                       double *est_out, double *dparam_out, double *G_dev, double *Gbar_dev, pt_stats *stats) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_grad: bad context/operator");
    PT_CHECK_ARG(col_dev && dparam_out, "pt_grad: NULL colour or dparam_out");
    PT_CHECK_ARG(n_colours >= 1 && n_sets >= 1 && set0 >= 0, "pt_grad: need n_colours, n_sets >= 1");
    PT_CHECK_ARG(mu >= 0 && mu < 4, "pt_grad: mu must be in 0..3");
    PT_CHECK_ARG(noise == PT_NOISE_Z2 || (noise == PT_NOISE_Z4 && op->dof == 12),
                 "pt_grad: Z4 noise needs the complex (Wilson) operator");
    PT_CHECK_ARG((G_dev == nullptr) == (Gbar_dev == nullptr), "pt_grad: pass both link outputs or neither");
    PT_CHECK_ARG(op->kind == 1 || G_dev == nullptr, "pt_grad: link gradients need the Wilson operator");
    int rc = check_solver_args(prec, tol, maxit);
    if (rc) return rc;
    PT_CUDA(cudaSetDevice(c->device));
    const int N = op->g.N;
    if (G_dev) {
        // [N][4][3][3] complex128 = 72 doubles per site
        PT_CUDA(cudaMemsetAsync(G_dev, 0, (size_t)N * 72 * sizeof(double), c->stream));
        PT_CUDA(cudaMemsetAsync(Gbar_dev, 0, (size_t)N * 72 * sizeof(double), c->stream));
    }
    std::vector<Task> all;
    build_probe_tasks(0, n_colours, set0, n_sets, op->dof, dilute, 1, all);
    const int n_pairs_total = (int)all.size() / 2;
    // chunk of pairs resident at once
    const int64_t L = pt_field_reals(op);
    const size_t per_slot = (size_t)L * (sizeof(double) + 7 * sizeof(double));
    int Q = (int)std::max<size_t>(1, std::min<size_t>((size_t)n_pairs_total, c->mem_budget / (2 * per_slot)));
    Q = std::min(Q, 512);
    double dparam_re = 0.0, dparam_im = 0.0;
    std::vector<double> est(n_sets * 2, 0.0);
    pt_stats acc;
    memset(&acc, 0, sizeof(acc));
    int rc_all = PT_OK;
    std::vector<double> part;
    for (int first = 0; first < n_pairs_total; first += Q) {
        const int np = std::min(Q, n_pairs_total - first);
        EngineRequest rq;
        rq.mode = MODE_GRAD;
        rq.n_tasks = 2 * np;
        rq.h_tasks = all.data() + 2 * first;
        rq.col = col_dev;
        rq.seed = seed;
        rq.noise = noise; rq.mu = mu; rq.n_p = 0; rq.dilute = dilute ? 1 : 0; rq.pshift = p;
        rq.p_list = nullptr;
        rq.B_user = nullptr;
        rq.X_user = nullptr;
        rq.tol = tol;
        rq.maxit = maxit;
        rq.prec = prec;
        rq.R_force = 2 * np;
        pt_stats st1;
        rc = run_engine(op, rq, &st1);
        if (rc != PT_OK && rc != PT_ERR_NOCONV) return rc;
        if (rc == PT_ERR_NOCONV) rc_all = rc;
        acc.n_rhs += st1.n_rhs; acc.inner_iters += st1.inner_iters; acc.outer_iters += st1.outer_iters;
        acc.site_rhs_applies += st1.site_rhs_applies; acc.engine_iters += st1.engine_iters;
        acc.graph_launches += st1.graph_launches; acc.kernel_launches += st1.kernel_launches;
        acc.max_relres = std::max(acc.max_relres, st1.max_relres); acc.n_slots = st1.n_slots;
        acc.n_noconv += st1.n_noconv;
        // the engine left x (slot 2i) and w (slot 2i+1) in its x64 buffer; rebuild its view
        EP P;
        memset(&P, 0, sizeof(P));
        P.g = op->g;
        P.nsb = (N + PT_BS - 1) / PT_BS;
        P.L = L;
        P.kappa = op->kappa;
        P.antip = op->antip;
        P.mode = MODE_GRAD;
        P.col = col_dev;
        P.seed = seed;
        P.noise = noise; P.mu = mu; P.dilute = dilute ? 1 : 0; P.pshift = p;
        P.x64 = rq.x64_out;
        Task *d_tasks = nullptr;
        PT_CUDA(cudaMallocAsync((void **)&d_tasks, (size_t)2 * np * sizeof(Task), c->stream));
        PT_CUDA(cudaMemcpyAsync(d_tasks, rq.h_tasks, (size_t)2 * np * sizeof(Task), cudaMemcpyHostToDevice, c->stream));
        P.tasks = d_tasks;
        double *d_part = nullptr;
        PT_CUDA(cudaMallocAsync((void **)&d_part, (size_t)np * P.nsb * 4 * sizeof(double), c->stream));
        if (op->kind == 0) k_grad_dots<0><<<c->num_sms * 8, PT_BS, 0, c->stream>>>(P, np, d_part);
        else k_grad_dots<1><<<c->num_sms * 8, PT_BS, 0, c->stream>>>(P, np, d_part);
        pt_kernel_launch_count += 2;
        if (G_dev) {
            int64_t n = (int64_t)N * 4;
            k_grad_links<<<(unsigned)((n + 127) / 128), 128, 0, c->stream>>>(P, np, G_dev, Gbar_dev);
            ++pt_kernel_launch_count;
        }
        PT_CUDA(cudaGetLastError());
        part.resize((size_t)np * P.nsb * 4);
        PT_CUDA(cudaMemcpyAsync(part.data(), d_part, part.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
        PT_CUDA(cudaFreeAsync(d_part, c->stream));
        PT_CUDA(cudaFreeAsync(d_tasks, c->stream));
        PT_CUDA(cudaStreamSynchronize(c->stream));
        for (int i = 0; i < np; ++i) {
            double yx_re = 0, yx_im = 0, yv_re = 0, yv_im = 0;
            for (int b = 0; b < P.nsb; ++b) {
                const double *q = &part[((size_t)i * P.nsb + b) * 4];
                yx_re += q[0]; yx_im += q[1]; yv_re += q[2]; yv_im += q[3];
            }
            // the estimate of this probe: v^H P A^{-1} v = (A^{-+} P^T v)^H v = y^H v
            const int s = all[2 * (first + i)].set - set0;
            est[2 * s] += yv_re;
            est[2 * s + 1] += yv_im;
            if (op->kind == 0) {          // dT/dm2 = - sum y^H x
                dparam_re -= yx_re;
                dparam_im -= yx_im;
            } else {                      // dT/dkappa = (1/kappa) sum (y^H x - y^H v)
                dparam_re += (yx_re - yv_re) / op->kappa;
                dparam_im += (yx_im - yv_im) / op->kappa;
            }
        }
    }
    dparam_out[0] = dparam_re;
    dparam_out[1] = dparam_im;
    if (est_out)
        for (int i = 0; i < 2 * n_sets; ++i) est_out[i] = est[i];
    if (stats) *stats = acc;
    return rc_all;
}

// ------------------------------------------------------------------ autotuner
// Coordinate descent over the engine's free parameters on a trial subset of
// the probes: even-odd or full system (every side even), the inner relative
// tolerance delta (mixed precision only), the right-hand sides per item and
// the slot group of the item order (Wilson only), the item shape (CTA threads;
// sites per thread for the Laplacian) and the engine iterations per CUDA
// graph.  Each candidate solves the same trial right-hand sides; the
// fastest (device time, synchronised) wins and is stored for the operator's
// (kind, precision, lattice).
static int store_tuning(pt_ctx *c, const pt_op *op, int prec, const pt_tune *t) {
    int slot = -1;
    for (int i = 0; i < 16; ++i) {
        pt_ctx::Tune &e = c->tune[i];
        if (e.used && e.kind == op->kind && e.prec == prec && !memcmp(e.dims, op->dims, sizeof(e.dims))) { slot = i; break; }
        if (!e.used && slot < 0) slot = i;
    }
    if (slot < 0) slot = 0;
    pt_ctx::Tune &e = c->tune[slot];
    if (!t) { e.used = 0; return PT_OK; }
    e.used = 1;
    e.kind = op->kind;
    e.prec = prec;
    memcpy(e.dims, op->dims, sizeof(e.dims));
    e.delta = t->delta;
    e.group = t->group;
    e.graph_iters = t->graph_iters;
    e.rhs_block = (t->rhs_block == 2 || t->rhs_block == WEO_G) ? t->rhs_block : 1;
    e.overlap = t->overlap ? 1 : 0;
    e.evenodd = t->evenodd ? 1 : 0;
    e.cta_threads = t->cta_threads;
    e.sites_per_thread = t->sites_per_thread;
    return PT_OK;
}

extern "C" int pt_set_tuning(pt_ctx *c, const pt_op *op, int prec, const pt_tune *t) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_set_tuning: bad context/operator");
    PT_CHECK_ARG(prec == PT_PREC_FP64 || prec == PT_PREC_MIXED_FP32 || prec == PT_PREC_MIXED_BF16,
                 "pt_set_tuning: unknown precision %d", prec);
    if (t) {
        PT_CHECK_ARG(t->delta >= 0.0 && t->delta < 1.0, "pt_set_tuning: delta must be in [0, 1)");
        PT_CHECK_ARG(t->group >= 1 && t->group <= 64, "pt_set_tuning: group must be in [1, 64]");
        PT_CHECK_ARG(t->graph_iters >= 1 && t->graph_iters <= 64, "pt_set_tuning: graph_iters must be in [1, 64]");
        PT_CHECK_ARG((t->rhs_block >= 0 && t->rhs_block <= 2) || t->rhs_block == WEO_G,
                     "pt_set_tuning: rhs_block must be 0, 1, 2 or %d", WEO_G);
        PT_CHECK_ARG(t->overlap == 0 || t->overlap == 1, "pt_set_tuning: overlap must be 0 or 1");
        PT_CHECK_ARG(t->evenodd == 0 || t->evenodd == 1, "pt_set_tuning: evenodd must be 0 or 1");
        PT_CHECK_ARG(t->cta_threads == 0 || t->cta_threads == 64 || t->cta_threads == 128 || t->cta_threads == 256,
                     "pt_set_tuning: cta_threads must be 0 (default), 64, 128 or 256");
        PT_CHECK_ARG(t->sites_per_thread == 0 || t->sites_per_thread == 4 || t->sites_per_thread == 8 ||
                         t->sites_per_thread == 16,
                     "pt_set_tuning: sites_per_thread must be 0 (default), 4, 8 or 16");
    }
    return store_tuning(c, op, prec, t);
}

extern "C" int pt_get_tuning(pt_ctx *c, const pt_op *op, int prec, pt_tune *t) {
    PT_CHECK_ARG(c && op && op->ctx == c && t, "pt_get_tuning: NULL argument");
    const pt_ctx::Tune e = engine_tuning(c, op, prec);
    t->delta = e.delta;
    t->group = e.group;
    t->graph_iters = e.graph_iters;
    t->rhs_block = e.rhs_block;
    t->overlap = e.overlap;
    t->evenodd = e.evenodd;
    t->cta_threads = e.cta_threads ? e.cta_threads : PT_BLOCK;
    t->sites_per_thread = op->kind ? 1 : (e.sites_per_thread ? e.sites_per_thread : Tile<0>::SPT);
    t->seconds_per_rhs = 0.0;
    return PT_OK;
}

extern "C" int pt_autotune(pt_ctx *c, const pt_op *op, const int32_t *col_dev, int n_colours, int mu, int noise,
                           uint64_t seed, int prec, double tol, int maxit, int trial_rhs, pt_tune *best) {
    PT_CHECK_ARG(c && op && op->ctx == c && col_dev && best, "pt_autotune: NULL argument");
    PT_CHECK_ARG(n_colours >= 1 && mu >= 0 && mu < 4 && trial_rhs >= 1, "pt_autotune: bad colours/mu/trial_rhs");
    PT_CHECK_ARG(noise == PT_NOISE_Z2 || (noise == PT_NOISE_Z4 && op->dof == 12),
                 "pt_autotune: Z4 noise needs the complex (Wilson) operator");
    int rc = check_solver_args(prec, tol, maxit);
    if (rc) return rc;
    PT_CUDA(cudaSetDevice(c->device));
    // trial tasks spread evenly over the colours and components of one noise set
    std::vector<Task> all, trial;
    build_probe_tasks(0, n_colours, 0, 1, op->dof, 1, 0, all);
    const int n = std::min<int>(trial_rhs, (int)all.size());
    for (int i = 0; i < n; ++i) trial.push_back(all[(size_t)i * all.size() / n]);
    const int p0 = 0;
    cudaEvent_t e0, e1;
    PT_CUDA(cudaEventCreate(&e0));
    PT_CUDA(cudaEventCreate(&e1));
    auto time_candidate = [&](const pt_ctx::Tune &cand, double *sec) -> int {
        EngineRequest rq;
        rq.mode = MODE_TRACE;
        rq.n_tasks = (int)trial.size();
        rq.h_tasks = trial.data();
        rq.col = col_dev;
        rq.seed = seed;
        rq.noise = noise; rq.mu = mu; rq.n_p = 1; rq.dilute = 1; rq.pshift = 0;
        rq.p_list = &p0;
        rq.B_user = nullptr;
        rq.X_user = nullptr;
        rq.tol = tol;
        rq.maxit = maxit;
        rq.prec = prec;
        rq.R_force = 0;
        c->trial = cand;
        c->in_trial = 1;
        cudaEventRecord(e0, c->stream);
        int r = run_engine(op, rq, nullptr);
        cudaEventRecord(e1, c->stream);
        c->in_trial = 0;
        if (r != PT_OK) return r;
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *sec = ms / 1e3;
        return PT_OK;
    };
    c->in_trial = 0;
    pt_ctx::Tune cur = engine_tuning(c, op, prec);
    double t_best = 0.0;
    rc = time_candidate(cur, &t_best);                       // warm-up (work space, first graph)
    if (!rc) rc = time_candidate(cur, &t_best);
    std::vector<double> deltas;
    if (prec == PT_PREC_MIXED_FP32) deltas = {1e-2, 1e-3, 1e-4, 1e-5, 1e-6};
    else if (prec == PT_PREC_MIXED_BF16) deltas = {3e-2, 1e-2, 3e-3, 1e-3};
    std::vector<int> groups;
    if (op->kind == 1) groups = {1, 2, 4, 8, 16};
    const std::vector<int> iters = {4, 8, 16};
    std::vector<int> blocks;
    if (op->kind == 1 && prec != PT_PREC_FP64 && op->csw == 0.0) blocks = {1, 2, WEO_G};
    std::vector<int> evenodds;
    if (pt_evenodd_ok(op->dims) && op->csw == 0.0) evenodds = {0, 1};     // the clover operator: even-odd only
    // item shape: CTA threads, and (Laplacian) sites per thread
    const std::vector<int> ctas = {64, 128, 256};
    std::vector<int> spts;
    if (op->kind == 0) spts = {4, 8, 16};
    // serial versus branched iterations (overlap) is left out: within 1 % either way, and the
    // branches blur the per-kernel event timing
    const std::vector<int> overlaps = {};
    for (int pass = 0; pass < 8 && !rc; ++pass) {
        const size_t nc = pass == 0 ? evenodds.size() : pass == 1 ? deltas.size() : pass == 2 ? blocks.size()
                          : pass == 3 ? groups.size() : pass == 4 ? ctas.size() : pass == 5 ? spts.size()
                          : pass == 6 ? iters.size() : overlaps.size();
        for (size_t i = 0; i < nc && !rc; ++i) {
            pt_ctx::Tune cand = cur;
            if (pass == 0) cand.evenodd = evenodds[i];
            else if (pass == 1) cand.delta = deltas[i];
            else if (pass == 2) cand.rhs_block = blocks[i];
            else if (pass == 3) cand.group = groups[i];
            else if (pass == 4) cand.cta_threads = ctas[i] == PT_BLOCK && !cur.cta_threads ? 0 : ctas[i];
            else if (pass == 5) cand.sites_per_thread = spts[i] == Tile<0>::SPT && !cur.sites_per_thread ? 0 : spts[i];
            else if (pass == 6) cand.graph_iters = iters[i];
            else cand.overlap = overlaps[i];
            if (!memcmp(&cand, &cur, sizeof(cand))) continue;
            double t = 0.0;
            rc = time_candidate(cand, &t);
            if (!rc && t < t_best) { t_best = t; cur = cand; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    c->in_trial = 0;
    if (rc) return rc;
    best->delta = cur.delta;
    best->group = cur.group;
    best->graph_iters = cur.graph_iters;
    best->rhs_block = cur.rhs_block;
    best->overlap = cur.overlap;
    best->evenodd = cur.evenodd;
    best->cta_threads = cur.cta_threads ? cur.cta_threads : PT_BLOCK;
    best->sites_per_thread = op->kind ? 1 : (cur.sites_per_thread ? cur.sites_per_thread : Tile<0>::SPT);
    best->seconds_per_rhs = t_best / trial.size();
    return store_tuning(c, op, prec, best);
}
