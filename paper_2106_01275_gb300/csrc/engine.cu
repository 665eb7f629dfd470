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
};

struct TaskStat {
    int iters, outer;
    double relres;
};

struct EP {
    Geom g;
    int kind, nsb, R;
    int64_t L;                 // reals per slot field
    double diag, kappa;
    int antip;
    const void *U;             // links in the inner precision
    const double *U64;         // links in FP64
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
    void *e, *r, *pv, *q, *s, *t, *r0;
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
#pragma unroll
        for (int s = 0; s < 4; ++s)
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                Cx<R> v = ld_cx<S, R>(f, P.g.N, 3 * s + a, idx);
                out[3 * s + a] = csub(v, cscale(acc[s][a], (R)P.kappa));
            }
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
    if (P.col[src] != tk.colour) return Cx<double>{0.0, 0.0};
    Cx<double> z;
    if (P.dilute) {
        if (a != tk.comp) return Cx<double>{0.0, 0.0};
        z = pt_noise(key, (uint64_t)src, P.noise);
    } else {
        z = pt_noise(key, (uint64_t)src * dof + a, P.noise);
    }
    return Cx<double>{sg * z.re, sg * z.im};
}

// ------------------------------------------------------------------ reduction tail
// Item partials -> (last item of the slot) deterministic total in `tot` (valid in
// all threads).  Returns true in every thread of the CTA that finishes the slot.
template <int K>
__device__ __forceinline__ bool slot_reduce(const EP &P, int j, int b, double v[K], double *sh, double tot[K]) {
    __shared__ int s_last;
    block_sum<K>(v, sh);
    if (threadIdx.x == 0) {
        double *dst = P.partials + ((size_t)j * P.nsb + b) * K;
#pragma unroll
        for (int k = 0; k < K; ++k) dst[k] = v[k];
        __threadfence();
        int prev = atomicAdd(&P.counters[j], 1);
        s_last = (prev == P.nsb - 1);
    }
    __syncthreads();
    bool last = s_last;
    if (last) {
        __threadfence();
        double acc[K];
#pragma unroll
        for (int k = 0; k < K; ++k) acc[k] = 0.0;
        const double *src = P.partials + (size_t)j * P.nsb * K;
        for (int i = threadIdx.x; i < P.nsb; i += blockDim.x)
#pragma unroll
            for (int k = 0; k < K; ++k) acc[k] += __ldcg(src + (size_t)i * K + k);
        block_sum<K>(acc, sh);
        if (threadIdx.x == 0) {
#pragma unroll
            for (int k = 0; k < K; ++k) sh[k] = acc[k];
            P.counters[j] = 0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < K; ++k) tot[k] = sh[k];
    }
    __syncthreads();
    return last;
}

// work-item loop helper: item -> (slot, site block); site-block-major order so
// that consecutive CTAs share a site block (link and halo reuse in L2)
#define ITEM_LOOP(LIST)                                                         \
    const int cnt = P.counts[LIST];                                             \
    const int *lst = P.lists + (size_t)(LIST) * P.R;                            \
    const int64_t n_items = (int64_t)cnt * P.nsb;                               \
    for (int64_t it = blockIdx.x; it < n_items; it += gridDim.x) {              \
        const int b = (int)(it / cnt);                                          \
        const int j = lst[it % cnt];

#define ITEM_LOOP_END }

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
        int in_i = (ph == PH_START || ph == PH_OUTER || ph == PH_INNER);
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
template <int KIND>
__global__ void __launch_bounds__(PT_BS) k_contract(EP P) {
    __shared__ double sh[32 * 2 * PT_MAX_P];
    const int N = P.g.N;
    ITEM_LOOP(LIST_CONTRACT)
        Slot &st = P.slots[j];
        if (st.phase != PH_CONTRACT) continue;
        const Task tk = P.tasks[st.task];
        const int idx = b * PT_BS + threadIdx.x;
        const double *x = P.x64 + (size_t)j * P.L;
        if (P.mode == MODE_SOLVE) {
            if (idx < N) {
                if constexpr (KIND == 0) {
                    P.X_user[(size_t)tk.set * N + idx] = x[idx];
                } else {
                    double *dst = P.X_user + ((size_t)tk.set * N + idx) * 24;
                    for (int c = 0; c < 12; ++c) {
                        Cx<double> v = ld_cx<double, double>(x, N, c, idx);
                        dst[2 * c] = v.re; dst[2 * c + 1] = v.im;
                    }
                }
            }
            double v[1] = {0.0}, tot[1];
            if (slot_reduce<1>(P, j, b, v, sh, tot) && threadIdx.x == 0) st.phase = PH_DONE;
            continue;
        }
        // trace mode: q_n = sum_x conj(v(x)) x(x + p_n e_mu), v = the task's probe
        double acc[2 * PT_MAX_P];
#pragma unroll
        for (int n = 0; n < 2 * PT_MAX_P; ++n) acc[n] = 0.0;
        if (idx < N && P.col[idx] == tk.colour) {
            int xc[4];
            site_coords(P.g, idx, xc);
            const uint64_t key = pt_set_key(P.seed, tk.set);
            const int dof = KIND ? 12 : 1;
            for (int a = 0; a < dof; ++a) {
                if (P.dilute && a != tk.comp) continue;
                Cx<double> z = P.dilute ? pt_noise(key, (uint64_t)idx, P.noise)
                                        : pt_noise(key, (uint64_t)idx * dof + a, P.noise);
#pragma unroll
                for (int n = 0; n < PT_MAX_P; ++n) {
                    if (n >= P.n_p) break;
                    int y = shift_site(P.g, idx, xc, P.mu, P.p[n]);
                    Cx<double> xv = Fld<KIND, double>::ld(x, N, a, y);
                    Cx<double> q = cconjmul(z, xv);
                    acc[2 * n] += q.re;
                    acc[2 * n + 1] += q.im;
                }
            }
        }
        double tot[2 * PT_MAX_P];
        if (slot_reduce<2 * PT_MAX_P>(P, j, b, acc, sh, tot) && threadIdx.x == 0) {
            for (int n = 0; n < P.n_p; ++n) {
                P.task_out[((size_t)st.task * P.n_p + n) * 2] = tot[2 * n];
                P.task_out[((size_t)st.task * P.n_p + n) * 2 + 1] = tot[2 * n + 1];
            }
            st.phase = PH_DONE;
        }
    ITEM_LOOP_END
}

// ------------------------------------------------------------------ outer (FP64) steps
template <int KIND, typename S>
__global__ void __launch_bounds__(PT_BS) k_outer_update(EP P) {
    typedef Fld<KIND, S> F;
    const int N = P.g.N;
    ITEM_LOOP(LIST_OUTER)
        const int ph = P.slots[j].phase;
        const int idx = b * PT_BS + threadIdx.x;
        if (idx >= N) continue;
        double *x = P.x64 + (size_t)j * P.L;
        const S *e = slot_cptr<S>(P.e, j, P.L);
        for (int c = 0; c < F::NC; ++c) {
            Cx<double> v = {0.0, 0.0};
            if (ph == PH_OUTER) {
                Cx<double> xv = Fld<KIND, double>::ld(x, N, c, idx);
                auto ev = F::ld(e, N, c, idx);
                v = Cx<double>{xv.re + (double)ev.re, xv.im + (double)ev.im};
            }
            Fld<KIND, double>::st(x, N, c, idx, v);
        }
    ITEM_LOOP_END
}

template <int KIND, typename S>
__global__ void __launch_bounds__(PT_BS) k_outer_residual(EP P) {
    typedef Fld<KIND, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 3];
    const int N = P.g.N;
    ITEM_LOOP(LIST_OUTER)
        Slot &st = P.slots[j];
        const int ph = st.phase;
        if (ph != PH_START && ph != PH_OUTER) continue;
        const Task tk = P.tasks[st.task];
        const int idx = b * PT_BS + threadIdx.x;
        double v[3] = {0.0, 0.0, 0.0};
        if (idx < N) {
            int xc[4];
            site_coords(P.g, idx, xc);
            const uint64_t key = (P.mode == MODE_SOLVE) ? 0 : pt_set_key(P.seed, tk.set);
            Cx<double> ax[F::NC];
            if (ph == PH_OUTER) {
                apply_site<KIND, double, double, double>(P, P.x64 + (size_t)j * P.L, P.U64, idx, xc, ax);
            } else {
#pragma unroll
                for (int c = 0; c < F::NC; ++c) ax[c] = Cx<double>{0.0, 0.0};
            }
            S *r = slot_ptr<S>(P.r, j, P.L);
            S *pv = slot_ptr<S>(P.pv, j, P.L);
            S *e = slot_ptr<S>(P.e, j, P.L);
            S *r0 = KIND ? slot_ptr<S>(P.r0, j, P.L) : nullptr;
            for (int c = 0; c < F::NC; ++c) {
                Cx<double> bv = source_val<KIND>(P, tk, key, idx, xc, c);
                Cx<double> rv = csub(bv, ax[c]);
                v[0] += rv.re * rv.re + rv.im * rv.im;
                v[1] += bv.re * bv.re + bv.im * bv.im;
                Cx<R> rs = Cx<R>{(R)rv.re, (R)rv.im};
                F::st(r, N, c, idx, rs);
                F::st(pv, N, c, idx, rs);
                if constexpr (KIND == 1) F::st(r0, N, c, idx, rs);
                F::st(e, N, c, idx, Cx<R>{R(0), R(0)});
                Cx<R> back = F::ld(r, N, c, idx);          // the inner solve sees the rounded r
                v[2] += (double)back.re * (double)back.re + (double)back.im * (double)back.im;
            }
        }
        double tot[3];
        if (slot_reduce<3>(P, j, b, v, sh, tot) && threadIdx.x == 0) {
            if (ph == PH_START) st.bnorm2 = tot[1];
            const double b2 = st.bnorm2;
            const double rel = b2 > 0.0 ? sqrt(tot[0] / b2) : 0.0;
            st.relres = rel;
            st.outer_it += 1;
            bool finite = isfinite(tot[0]);
            if (!finite) atomicOr(&P.flags[FLAG_NUMERIC], 1);
            bool conv = (b2 == 0.0) || rel <= P.tol;
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
                const double floor2 = 0.25 * P.tol * P.tol * b2;
                st.target2 = fmax(P.delta * P.delta * tot[2], floor2);
            }
        }
    ITEM_LOOP_END
}

// ------------------------------------------------------------------ CG (Laplacian)
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BS) k_cg_apply(EP P) {
    typedef Fld<0, S> F;
    typedef typename F::R R;
    __shared__ double sh[32];
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int idx = b * PT_BS + threadIdx.x;
        double v[1] = {0.0};
        if (idx < N) {
            int xc[4];
            site_coords(P.g, idx, xc);
            const S *pv = slot_cptr<S>(P.pv, j, P.L);
            R q = lap_site<R, S>(P.g, pv, (R)P.diag, idx, xc);
            st_real(slot_ptr<S>(P.q, j, P.L), (size_t)idx, q);
            v[0] = (double)ld_real(pv, (size_t)idx) * (double)q;
        }
        double tot[1];
        if (slot_reduce<1>(P, j, b, v, sh, tot) && threadIdx.x == 0) {
            if (!(tot[0] > 0.0) || !isfinite(tot[0])) {
                atomicOr(&P.flags[FLAG_NUMERIC], 2);
                st.phase = PH_OUTER;                     // fall back to a true-residual restart
                st.alpha = Cx<double>{0.0, 0.0};
            } else {
                st.alpha = Cx<double>{st.rr / tot[0], 0.0};
            }
        }
    ITEM_LOOP_END
}

template <typename S>
__global__ void __launch_bounds__(PT_BS) k_cg_update(EP P) {
    __shared__ double sh[32];
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int idx = b * PT_BS + threadIdx.x;
        double v[1] = {0.0};
        if (idx < N) {
            typedef typename ArithT<S>::T R;
            const R al = (R)st.alpha.re;
            S *e = slot_ptr<S>(P.e, j, P.L);
            S *r = slot_ptr<S>(P.r, j, P.L);
            const S *pv = slot_cptr<S>(P.pv, j, P.L);
            const S *q = slot_cptr<S>(P.q, j, P.L);
            R ev = ld_real(e, (size_t)idx) + al * ld_real(pv, (size_t)idx);
            R rv = ld_real(r, (size_t)idx) - al * ld_real(q, (size_t)idx);
            st_real(e, (size_t)idx, ev);
            st_real(r, (size_t)idx, rv);
            double rs = (double)ld_real(r, (size_t)idx);
            v[0] = rs * rs;
        }
        double tot[1];
        if (slot_reduce<1>(P, j, b, v, sh, tot) && threadIdx.x == 0) {
            st.inner_it += 1;
            st.total_it += 1;
            if (tot[0] <= st.target2 || st.inner_it >= P.max_inner || st.total_it >= P.maxit || !isfinite(tot[0])) {
                st.phase = PH_OUTER;
            } else {
                st.beta = Cx<double>{tot[0] / st.rr, 0.0};
                st.rr = tot[0];
            }
        }
    ITEM_LOOP_END
}

template <typename S>
__global__ void __launch_bounds__(PT_BS) k_cg_dir(EP P) {
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int idx = b * PT_BS + threadIdx.x;
        if (idx >= N) continue;
        typedef typename ArithT<S>::T R;
        const R be = (R)st.beta.re;
        S *pv = slot_ptr<S>(P.pv, j, P.L);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        st_real(pv, (size_t)idx, ld_real(r, (size_t)idx) + be * ld_real(pv, (size_t)idx));
    ITEM_LOOP_END
}

// ------------------------------------------------------------------ BiCGStab (Wilson)
// v = A p;  alpha = rho / (r0, v)
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BS) k_bicg_apply1(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 2];
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int idx = b * PT_BS + threadIdx.x;
        double v[2] = {0.0, 0.0};
        if (idx < N) {
            int xc[4];
            site_coords(P.g, idx, xc);
            Cx<R> av[12];
            apply_site<1, R, S, LS>(P, slot_cptr<S>(P.pv, j, P.L), (const LS *)P.U, idx, xc, av);
            S *q = slot_ptr<S>(P.q, j, P.L);
            const S *r0 = slot_cptr<S>(P.r0, j, P.L);
            for (int c = 0; c < 12; ++c) {
                F::st(q, N, c, idx, av[c]);
                Cx<R> w = F::ld(q, N, c, idx);
                Cx<R> z = F::ld(r0, N, c, idx);
                v[0] += (double)z.re * w.re + (double)z.im * w.im;
                v[1] += (double)z.re * w.im - (double)z.im * w.re;
            }
        }
        double tot[2];
        if (slot_reduce<2>(P, j, b, v, sh, tot) && threadIdx.x == 0) {
            double d2 = tot[0] * tot[0] + tot[1] * tot[1];
            if (!(d2 > 0.0) || !isfinite(d2)) {
                atomicOr(&P.flags[FLAG_NUMERIC], 4);
                st.phase = PH_OUTER;
                st.alpha = Cx<double>{0.0, 0.0};
            } else {
                // alpha = rho / (r0, v)
                st.alpha = Cx<double>{(st.rho.re * tot[0] + st.rho.im * tot[1]) / d2,
                                      (st.rho.im * tot[0] - st.rho.re * tot[1]) / d2};
            }
        }
    ITEM_LOOP_END
}

// s = r - alpha v
template <typename S>
__global__ void __launch_bounds__(PT_BS) k_bicg_s(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int idx = b * PT_BS + threadIdx.x;
        if (idx >= N) continue;
        const Cx<R> al = Cx<R>{(R)st.alpha.re, (R)st.alpha.im};
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *q = slot_cptr<S>(P.q, j, P.L);
        S *s = slot_ptr<S>(P.s, j, P.L);
        for (int c = 0; c < 12; ++c) F::st(s, N, c, idx, csub(F::ld(r, N, c, idx), cmul(al, F::ld(q, N, c, idx))));
    ITEM_LOOP_END
}

// t = A s;  omega = (t, s) / (t, t)
template <typename S, typename LS>
__global__ void __launch_bounds__(PT_BS) k_bicg_apply2(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 3];
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int idx = b * PT_BS + threadIdx.x;
        double v[3] = {0.0, 0.0, 0.0};
        if (idx < N) {
            int xc[4];
            site_coords(P.g, idx, xc);
            Cx<R> av[12];
            const S *s = slot_cptr<S>(P.s, j, P.L);
            apply_site<1, R, S, LS>(P, s, (const LS *)P.U, idx, xc, av);
            S *t = slot_ptr<S>(P.t, j, P.L);
            for (int c = 0; c < 12; ++c) {
                F::st(t, N, c, idx, av[c]);
                Cx<R> tv = F::ld(t, N, c, idx);
                Cx<R> sv = F::ld(s, N, c, idx);
                v[0] += (double)tv.re * sv.re + (double)tv.im * sv.im;     // (t, s) = conj(t) s
                v[1] += (double)tv.re * sv.im - (double)tv.im * sv.re;
                v[2] += (double)tv.re * tv.re + (double)tv.im * tv.im;
            }
        }
        double tot[3];
        if (slot_reduce<3>(P, j, b, v, sh, tot) && threadIdx.x == 0) {
            if (!(tot[2] > 0.0) || !isfinite(tot[2])) {
                st.omega = Cx<double>{0.0, 0.0};
            } else {
                st.omega = Cx<double>{tot[0] / tot[2], tot[1] / tot[2]};
            }
        }
    ITEM_LOOP_END
}

// e += alpha p + omega s;  r = s - omega t;  rho' = (r0, r), |r|^2
template <typename S>
__global__ void __launch_bounds__(PT_BS) k_bicg_update(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    __shared__ double sh[32 * 3];
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int idx = b * PT_BS + threadIdx.x;
        double v[3] = {0.0, 0.0, 0.0};
        if (idx < N) {
            const Cx<R> al = Cx<R>{(R)st.alpha.re, (R)st.alpha.im};
            const Cx<R> om = Cx<R>{(R)st.omega.re, (R)st.omega.im};
            S *e = slot_ptr<S>(P.e, j, P.L);
            S *r = slot_ptr<S>(P.r, j, P.L);
            const S *pv = slot_cptr<S>(P.pv, j, P.L);
            const S *s = slot_cptr<S>(P.s, j, P.L);
            const S *t = slot_cptr<S>(P.t, j, P.L);
            const S *r0 = slot_cptr<S>(P.r0, j, P.L);
            for (int c = 0; c < 12; ++c) {
                Cx<R> sv = F::ld(s, N, c, idx);
                F::st(e, N, c, idx, cadd(F::ld(e, N, c, idx), cadd(cmul(al, F::ld(pv, N, c, idx)), cmul(om, sv))));
                F::st(r, N, c, idx, csub(sv, cmul(om, F::ld(t, N, c, idx))));
                Cx<R> rv = F::ld(r, N, c, idx);
                Cx<R> z = F::ld(r0, N, c, idx);
                v[0] += (double)z.re * rv.re + (double)z.im * rv.im;
                v[1] += (double)z.re * rv.im - (double)z.im * rv.re;
                v[2] += (double)rv.re * rv.re + (double)rv.im * rv.im;
            }
        }
        double tot[3];
        if (slot_reduce<3>(P, j, b, v, sh, tot) && threadIdx.x == 0) {
            st.inner_it += 1;
            st.total_it += 1;
            const double om2 = st.omega.re * st.omega.re + st.omega.im * st.omega.im;
            const double rho2 = st.rho.re * st.rho.re + st.rho.im * st.rho.im;
            if (tot[2] <= st.target2 || st.inner_it >= P.max_inner || st.total_it >= P.maxit ||
                !isfinite(tot[2]) || !(om2 > 0.0) || !(rho2 > 0.0)) {
                st.phase = PH_OUTER;
            } else {
                // beta = (rho' / rho) (alpha / omega)
                Cx<double> rn = Cx<double>{tot[0], tot[1]};
                Cx<double> q1 = Cx<double>{(rn.re * st.rho.re + rn.im * st.rho.im) / rho2,
                                           (rn.im * st.rho.re - rn.re * st.rho.im) / rho2};
                Cx<double> q2 = Cx<double>{(st.alpha.re * st.omega.re + st.alpha.im * st.omega.im) / om2,
                                           (st.alpha.im * st.omega.re - st.alpha.re * st.omega.im) / om2};
                st.beta = cmul(q1, q2);
                st.rho = rn;
                st.rr = tot[2];
            }
        }
    ITEM_LOOP_END
}

// p = r + beta (p - omega v)
template <typename S>
__global__ void __launch_bounds__(PT_BS) k_bicg_dir(EP P) {
    typedef Fld<1, S> F;
    typedef typename F::R R;
    const int N = P.g.N;
    ITEM_LOOP(LIST_INNER)
        const Slot &st = P.slots[j];
        if (st.phase != PH_INNER) continue;
        const int idx = b * PT_BS + threadIdx.x;
        if (idx >= N) continue;
        const Cx<R> be = Cx<R>{(R)st.beta.re, (R)st.beta.im};
        const Cx<R> om = Cx<R>{(R)st.omega.re, (R)st.omega.im};
        S *pv = slot_ptr<S>(P.pv, j, P.L);
        const S *r = slot_cptr<S>(P.r, j, P.L);
        const S *q = slot_cptr<S>(P.q, j, P.L);
        for (int c = 0; c < 12; ++c) {
            Cx<R> pp = csub(F::ld(pv, N, c, idx), cmul(om, F::ld(q, N, c, idx)));
            F::st(pv, N, c, idx, cadd(F::ld(r, N, c, idx), cmul(be, pp)));
        }
    ITEM_LOOP_END
}

// ------------------------------------------------------------------ host driver
struct EngineRun {
    EP P;
    int grid_items;
    int kernels_per_iter;
};

template <int KIND, typename S, typename LS>
static void enqueue_iteration(const EngineRun &E, cudaStream_t st) {
    const EP &P = E.P;
    const int G = E.grid_items;
    k_schedule<<<1, 1024, 0, st>>>(P);
    k_contract<KIND><<<G, PT_BS, 0, st>>>(P);
    k_outer_update<KIND, S><<<G, PT_BS, 0, st>>>(P);
    k_outer_residual<KIND, S><<<G, PT_BS, 0, st>>>(P);
    if constexpr (KIND == 0) {
        k_cg_apply<S, LS><<<G, PT_BS, 0, st>>>(P);
        k_cg_update<S><<<G, PT_BS, 0, st>>>(P);
        k_cg_dir<S><<<G, PT_BS, 0, st>>>(P);
    } else {
        k_bicg_apply1<S, LS><<<G, PT_BS, 0, st>>>(P);
        k_bicg_s<S><<<G, PT_BS, 0, st>>>(P);
        k_bicg_apply2<S, LS><<<G, PT_BS, 0, st>>>(P);
        k_bicg_update<S><<<G, PT_BS, 0, st>>>(P);
        k_bicg_dir<S><<<G, PT_BS, 0, st>>>(P);
    }
}

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
    // outputs
    std::vector<double> task_out;   // trace: [n_tasks][n_p] complex
    std::vector<TaskStat> tstat;
    double *x64_out;           // grad mode: device pointer to the solutions (valid until next call)
    int R_used;
};

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

template <int KIND, typename S, typename LS>
static int run_engine_t(const pt_op *op, EngineRequest &rq, pt_stats *stats) {
    pt_ctx *c = op->ctx;
    const Geom g = op->g;
    const int64_t L = pt_field_reals(op);
    const int nvec = KIND ? 7 : 4;
    const size_t per_slot = (size_t)L * (sizeof(double) + nvec * sizeof(S));
    int R = rq.R_force > 0 ? rq.R_force : (int)std::min<size_t>((size_t)rq.n_tasks, c->mem_budget / per_slot);
    if (R < 1) R = 1;
    if (rq.R_force <= 0) R = std::min(R, 4096);
    const int nsb = (g.N + PT_BS - 1) / PT_BS;
    const int K_MAX = 2 * PT_MAX_P;
    // layout of the work space
    size_t off = 0;
    auto take = [&](size_t bytes) { size_t o = off; off += align256(bytes); return o; };
    size_t o_x64 = take((size_t)R * L * sizeof(double));
    size_t o_vec[7];
    for (int v = 0; v < nvec; ++v) o_vec[v] = take((size_t)R * L * sizeof(S));
    size_t o_slots = take((size_t)R * sizeof(Slot));
    size_t o_part = take((size_t)R * nsb * K_MAX * sizeof(double));
    size_t o_cnt = take((size_t)R * sizeof(int));
    size_t o_lists = take((size_t)3 * R * sizeof(int));
    size_t o_counts = take(4 * sizeof(int));
    size_t o_head = take(sizeof(int));
    size_t o_flags = take(8 * sizeof(int));
    size_t o_tasks = take((size_t)rq.n_tasks * sizeof(Task));
    size_t o_tstat = take((size_t)rq.n_tasks * sizeof(TaskStat));
    size_t o_tout = take((size_t)rq.n_tasks * std::max(rq.n_p, 1) * 2 * sizeof(double));
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
    P.R = R;
    P.L = L;
    P.diag = 8.0 + op->m2;
    P.kappa = op->kappa;
    P.antip = op->antip;
    if constexpr (KIND == 1) {
        P.U = std::is_same<S, double>::value ? (const void *)op->U64
              : std::is_same<S, float>::value ? (const void *)op->U32 : (const void *)op->U16;
    }
    P.U64 = op->U64;
    P.mode = rq.mode;
    P.col = rq.col;
    P.seed = rq.seed;
    P.noise = rq.noise;
    P.mu = rq.mu;
    P.n_p = rq.n_p;
    P.dilute = rq.dilute;
    P.pshift = rq.pshift;
    for (int n = 0; n < rq.n_p && n < PT_MAX_P; ++n) P.p[n] = rq.p_list[n];
    P.tasks = (const Task *)(base + o_tasks);
    P.n_tasks = rq.n_tasks;
    P.B_user = rq.B_user;
    P.X_user = rq.X_user;
    P.x64 = (double *)(base + o_x64);
    void **vp[7] = {&P.e, &P.r, &P.pv, &P.q, &P.s, &P.t, &P.r0};
    for (int v = 0; v < nvec; ++v) *vp[v] = base + o_vec[v];
    P.slots = (Slot *)(base + o_slots);
    P.partials = (double *)(base + o_part);
    P.counters = (int *)(base + o_cnt);
    P.lists = (int *)(base + o_lists);
    P.counts = (int *)(base + o_counts);
    P.head = (int *)(base + o_head);
    P.flags = (int *)(base + o_flags);
    P.tstat = (TaskStat *)(base + o_tstat);
    P.task_out = (double *)(base + o_tout);
    P.tol = rq.tol;
    P.maxit = rq.maxit;
    if (rq.prec == PT_PREC_FP64) { P.delta = 0.0; P.max_inner = rq.maxit; }
    else if (rq.prec == PT_PREC_MIXED_FP32) { P.delta = KIND ? 1e-5 : 1e-5; P.max_inner = 4000; }
    else { P.delta = 1e-2; P.max_inner = 400; }

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

    int occ = 0;
    if constexpr (KIND == 0) {
        PT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_cg_apply<S, LS>, PT_BS, 0));
    } else {
        PT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_bicg_apply1<S, LS>, PT_BS, 0));
    }
    occ = std::max(occ, 1);
    E.grid_items = c->num_sms * occ;
    E.kernels_per_iter = KIND ? 9 : 7;

    // capture ITERS engine iterations into one graph
    const int ITERS = 8;
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    PT_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < ITERS; ++i) enqueue_iteration<KIND, S, LS>(E, c->cap_stream);
    cudaError_t ce = cudaStreamEndCapture(c->cap_stream, &graph);
    if (ce != cudaSuccess) return pt_cuda_fail(ce, "cudaStreamEndCapture", __FILE__, __LINE__);
    ce = cudaGraphInstantiate(&exec, graph, 0);
    if (ce != cudaSuccess) { cudaGraphDestroy(graph); return pt_cuda_fail(ce, "cudaGraphInstantiate", __FILE__, __LINE__); }

    // bounded host loop: every RHS stops within maxit Krylov iterations, plus a
    // few engine iterations per outer restart and per retire/refill
    const int64_t waves = (rq.n_tasks + R - 1) / R + 1;
    const int64_t max_launches = waves * ((int64_t)rq.maxit * 2 + 400) / ITERS + 64;
    int64_t launches = 0;
    int rc_loop = PT_OK;
    int *hf = c->h_flags;
    while (true) {
        ce = cudaGraphLaunch(exec, st);
        if (ce != cudaSuccess) { rc_loop = pt_cuda_fail(ce, "cudaGraphLaunch", __FILE__, __LINE__); break; }
        ++launches;
        ce = cudaMemcpyAsync(hf, P.flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, st);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
        if (ce != cudaSuccess) { rc_loop = pt_cuda_fail(ce, "engine flag read", __FILE__, __LINE__); break; }
        if (hf[FLAG_DONE]) break;
        if (launches >= max_launches) {
            pt_set_error("solver engine did not finish within %lld graph launches", (long long)max_launches);
            rc_loop = PT_ERR_TIMEOUT;
            break;
        }
    }
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
    for (int i = 0; i < nrhs; ++i) tasks[i] = Task{i, 0, 0, 0};
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
static void build_probe_tasks(int n_colours, int set0, int n_sets, int dof, int dilute, int adj_pairs,
                              std::vector<Task> &tasks) {
    tasks.clear();
    const int ncomp = dilute ? dof : 1;
    for (int s = 0; s < n_sets; ++s)
        for (int col = 0; col < n_colours; ++col)
            for (int a = 0; a < ncomp; ++a) {
                tasks.push_back(Task{set0 + s, col, dilute ? a : -1, 0});
                if (adj_pairs) tasks.push_back(Task{set0 + s, col, dilute ? a : -1, TASK_ADJ});
            }
}

extern "C" int pt_trace_PAinv(pt_ctx *c, const pt_op *op, const int32_t *col_dev, int n_colours, int mu,
                              const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets, int dilute,
                              int prec, double tol, int maxit, double *est_out, double *mean_out, double *var_out,
                              pt_stats *stats) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_trace_PAinv: bad context/operator");
    PT_CHECK_ARG(col_dev && est_out, "pt_trace_PAinv: NULL colour or output array");
    PT_CHECK_ARG(n_colours >= 1 && n_sets >= 1 && set0 >= 0, "pt_trace_PAinv: need n_colours, n_sets >= 1");
    PT_CHECK_ARG(mu >= 0 && mu < 4, "pt_trace_PAinv: mu must be in 0..3");
    PT_CHECK_ARG(n_p >= 1 && n_p <= PT_MAX_P && p_list, "pt_trace_PAinv: 1 <= n_p <= %d", PT_MAX_P);
    PT_CHECK_ARG(noise == PT_NOISE_Z2 || (noise == PT_NOISE_Z4 && op->dof == 12),
                 "pt_trace_PAinv: Z4 noise needs the complex (Wilson) operator");
    int rc = check_solver_args(prec, tol, maxit);
    if (rc) return rc;
    PT_CUDA(cudaSetDevice(c->device));
    std::vector<Task> tasks;
    build_probe_tasks(n_colours, set0, n_sets, op->dof, dilute, 0, tasks);
    EngineRequest rq;
    rq.mode = MODE_TRACE;
    rq.n_tasks = (int)tasks.size();
    rq.h_tasks = tasks.data();
    rq.col = col_dev;
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
    // per-set sums in a fixed task order (deterministic)
    for (int s = 0; s < n_sets; ++s)
        for (int n = 0; n < n_p; ++n) { est_out[(s * n_p + n) * 2] = 0.0; est_out[(s * n_p + n) * 2 + 1] = 0.0; }
    for (size_t t = 0; t < tasks.size(); ++t) {
        int s = tasks[t].set - set0;
        for (int n = 0; n < n_p; ++n) {
            est_out[(s * n_p + n) * 2] += rq.task_out[(t * n_p + n) * 2];
            est_out[(s * n_p + n) * 2 + 1] += rq.task_out[(t * n_p + n) * 2 + 1];
        }
    }
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
    build_probe_tasks(n_colours, set0, n_sets, op->dof, dilute, 1, all);
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
