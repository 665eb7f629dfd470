// Batched even-odd trace estimation for the shifted Laplacian (Eqs. (1), (5)
// with the solves on the Schur complement; the even-odd building blocks of
// evenodd.cu give the arithmetic).
//
// Every task (noise set s, colour c) solves A x = v, v(y) = Re z_s(y) [col(y) = c],
// through the even system S x_e = b'_e (S = d - H_eo H_oe / d, d = 8 + m^2,
// b'_e = v_e + H_eo v_o / d), and contributes
//   q_n = sum_{x : col(x) = c} conj(z_s(x)) x(x + p_n e_mu),
// with x on the odd sites rebuilt where it is read, x_o = (v_o + H_oe x_e) / d
// (the same sources and contraction as the batched engine's Laplacian trace).
// The tasks of a batch advance in lockstep: FP32 CG on the even sites (each
// task to its own inner tolerance) inside FP64 defect correction (the true
// residual b'_e - S x_e with b'_e regenerated from the noise), then the
// contraction.  Per-task scalars live on the host; each step ends with one
// per-task reduction (fixed summation order).
//
// The per-site arithmetic and the sequence of steps are shared by the device
// entry point and a host-only twin: only the loop over sites differs.
#include <algorithm>
#include <cmath>
#include <vector>

#include "eo_geom.cuh"
#include "hd_complex.cuh"
#include "pt_common.cuh"

struct ETP {
    EoGeom g;
    double d;               // 8 + m^2
    const int32_t *col;     // [N]
    uint64_t seed;
    int noise, mu, n_p, m;  // m colours
    int set0, t0;           // task t0 + r of the batch: set set0 + (t0 + r) / m, colour (t0 + r) % m
    int p[PT_MAX_P];
};

// SplitMix64 noise (the library's counter-based generator, Steele, Lea and
// Flood 2014): h = mix64(key + (c + 1) GAMMA); Z2 = 1 - 2 (h >> 63),
// Z4 = i^(h >> 62)
__host__ __device__ __forceinline__ zd et_noise(uint64_t key, uint64_t c, int kind) {
    const uint64_t h = pt_mix64(key + (c + 1ULL) * PT_GAMMA);
    if (kind == PT_NOISE_Z2) return {(h >> 63) ? -1.0 : 1.0, 0.0};
    switch ((int)(h >> 62)) {
        case 0: return {1.0, 0.0};
        case 1: return {0.0, 1.0};
        case 2: return {-1.0, 0.0};
        default: return {0.0, -1.0};
    }
}

struct ETTask {
    int colour;
    uint64_t key;
};

__host__ __device__ __forceinline__ ETTask et_task(const ETP &P, int r) {
    const int t = P.t0 + r;
    return ETTask{t % P.m, pt_set_key(P.seed, P.set0 + t / P.m)};
}

// the probe of a task at storage index y (real part of the noise)
__host__ __device__ __forceinline__ double et_b(const ETP &P, const ETTask &T, int y) {
    return P.col[y] == T.colour ? et_noise(T.key, (uint64_t)y, P.noise).re : 0.0;
}

// sum of the eight neighbours of entry h (parity par) read from a half field
// of the other parity
template <typename T>
__host__ __device__ __forceinline__ T et_nbsum(const EoGeom &g, int par, const T *src, int h) {
    int x[4];
    const int i = eo_full_site(g, par, h, x);
    T s = T(0);
    for (int mu = 0; mu < 4; ++mu) {
        s += src[eo_neighbour(g, i, x, mu, 1) >> 1];
        s += src[eo_neighbour(g, i, x, mu, -1) >> 1];
    }
    return s;
}

// b'_e at even entry h
__host__ __device__ __forceinline__ double et_bprime(const ETP &P, const ETTask &T, int h) {
    int x[4];
    const int i = eo_full_site(P.g, 0, h, x);
    double s = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
        s += et_b(P, T, eo_neighbour(P.g, i, x, mu, 1));
        s += et_b(P, T, eo_neighbour(P.g, i, x, mu, -1));
    }
    return et_b(P, T, i) + s / P.d;
}

// per-task fields of the batch, entry (r, h) at r Nh + h
struct ETF {
    double *x64, *t64;           // solution (even), H_oe x (odd)
    float *r, *p, *q, *e, *t;    // inner CG (even; t odd)
};

// outer step 1 at odd entry h: t64 = H_oe x64
__host__ __device__ __forceinline__ void et_outer1(const ETP &P, const ETF &F, int r, int h) {
    const size_t o = (size_t)r * P.g.Nh;
    F.t64[o + h] = et_nbsum(P.g, 1, F.x64 + o, h);
}

// outer step 2 at even entry h: r64 = b'_e - S x64; r = (float) r64, e = p = 0;
// adds |r64|^2, |b'|^2, |r|^2 to v
__host__ __device__ __forceinline__ void et_outer2(const ETP &P, const ETF &F, int r, int h, double v[3]) {
    const size_t o = (size_t)r * P.g.Nh;
    const ETTask T = et_task(P, r);
    const double bp = et_bprime(P, T, h);
    const double sx = P.d * F.x64[o + h] - et_nbsum(P.g, 0, F.t64 + o, h) / P.d;
    const double rv = bp - sx;
    const float rs = (float)rv;
    F.r[o + h] = rs;
    F.e[o + h] = 0.0f;
    F.p[o + h] = 0.0f;
    v[0] += rv * rv;
    v[1] += bp * bp;
    v[2] += (double)rs * (double)rs;
}

// inner step A at odd entry h: t = H_oe (r + beta p)
__host__ __device__ __forceinline__ void et_innerA(const ETP &P, const ETF &F, int r, int h, float beta) {
    const size_t o = (size_t)r * P.g.Nh;
    int x[4];
    const int i = eo_full_site(P.g, 1, h, x);
    float s = 0.0f;
    for (int mu = 0; mu < 4; ++mu)
        for (int dir = 0; dir < 2; ++dir) {
            const size_t k = o + (eo_neighbour(P.g, i, x, mu, dir ? -1 : 1) >> 1);
            s += F.r[k] + beta * F.p[k];
        }
    F.t[o + h] = s;
}

// inner step B at even entry h: p = r + beta p, q = S p = d p - H_eo t / d; adds p q
__host__ __device__ __forceinline__ void et_innerB(const ETP &P, const ETF &F, int r, int h, float beta,
                                                  double v[1]) {
    const size_t o = (size_t)r * P.g.Nh;
    const float pv = F.r[o + h] + beta * F.p[o + h];
    const float qv = (float)P.d * pv - et_nbsum(P.g, 0, F.t + o, h) / (float)P.d;
    F.p[o + h] = pv;
    F.q[o + h] = qv;
    v[0] += (double)pv * (double)qv;
}

// inner step C at even entry h: e += alpha p, r -= alpha q; adds r r
__host__ __device__ __forceinline__ void et_innerC(const ETP &P, const ETF &F, int r, int h, float alpha,
                                                  double v[1]) {
    const size_t o = (size_t)r * P.g.Nh;
    F.e[o + h] += alpha * F.p[o + h];
    const float rv = F.r[o + h] - alpha * F.q[o + h];
    F.r[o + h] = rv;
    v[0] += (double)rv * (double)rv;
}

// outer update at even entry h: x64 += e
__host__ __device__ __forceinline__ void et_update(const ETP &P, const ETF &F, int r, int h) {
    const size_t o = (size_t)r * P.g.Nh;
    F.x64[o + h] += (double)F.e[o + h];
}

// the full solution at storage index y: x_e, or x_o = (v_o + H_oe x_e) / d
__host__ __device__ __forceinline__ double et_x(const ETP &P, const ETF &F, const ETTask &T, int r, int y) {
    const size_t o = (size_t)r * P.g.Nh;
    int x[4], q = y, par = 0;
    for (int mu = 0; mu < 4; ++mu) { x[mu] = q % P.g.D[mu]; q /= P.g.D[mu]; par += x[mu]; }
    if ((par & 1) == 0) return F.x64[o + (y >> 1)];
    double s = 0.0;
    for (int mu = 0; mu < 4; ++mu) {
        s += F.x64[o + (eo_neighbour(P.g, y, x, mu, 1) >> 1)];
        s += F.x64[o + (eo_neighbour(P.g, y, x, mu, -1) >> 1)];
    }
    return (et_b(P, T, y) + s) / P.d;
}

// contraction at storage index i: v[2n], v[2n+1] += conj(z(i)) x(i + p_n e_mu)
// where col(i) = c
__host__ __device__ __forceinline__ void et_contract(const ETP &P, const ETF &F, int r, int i,
                                                    double v[2 * PT_MAX_P]) {
    const ETTask T = et_task(P, r);
    if (P.col[i] != T.colour) return;
    const zd z = et_noise(T.key, (uint64_t)i, P.noise);
    const int c_mu = (i / P.g.stride[P.mu]) % P.g.D[P.mu];
    for (int n = 0; n < P.n_p; ++n) {
        int cm = (c_mu + P.p[n]) % P.g.D[P.mu];
        if (cm < 0) cm += P.g.D[P.mu];
        const int y = i + (cm - c_mu) * P.g.stride[P.mu];
        const double xv = et_x(P, F, T, r, y);
        v[2 * n] += z.re * xv;
        v[2 * n + 1] -= z.im * xv;
    }
}

// ---------------------------------------------------------------- steps
enum { ET_OUTER1 = 0, ET_OUTER2, ET_INNERA, ET_INNERB, ET_INNERC, ET_UPDATE, ET_CONTRACT };

// reduced values per task, and the sites a step runs over (half fields; the
// contraction runs over the whole lattice)
__host__ __device__ __forceinline__ int et_k(int step, int n_p) {
    return step == ET_OUTER2 ? 3 : (step == ET_INNERB || step == ET_INNERC) ? 1 : step == ET_CONTRACT ? 2 * n_p : 0;
}

template <int STEP>
__host__ __device__ __forceinline__ void et_site(const ETP &P, const ETF &F, int r, int idx, float coef, double *v) {
    if constexpr (STEP == ET_OUTER1) et_outer1(P, F, r, idx);
    else if constexpr (STEP == ET_OUTER2) et_outer2(P, F, r, idx, v);
    else if constexpr (STEP == ET_INNERA) et_innerA(P, F, r, idx, coef);
    else if constexpr (STEP == ET_INNERB) et_innerB(P, F, r, idx, coef, v);
    else if constexpr (STEP == ET_INNERC) et_innerC(P, F, r, idx, coef, v);
    else if constexpr (STEP == ET_UPDATE) et_update(P, F, r, idx);
    else et_contract(P, F, r, idx, v);
}

#define ET_NT 256
#define ET_KMAX (2 * PT_MAX_P)

// grid (site blocks, tasks): block b of task r; partials[(r nblk + b) K + k]
template <int STEP>
__global__ void __launch_bounds__(ET_NT) k_et_step(ETP P, ETF F, const int *act, const float *coef, int nsites,
                                                   int nblk, double *partials) {
    __shared__ double sh[ET_NT / 32][ET_KMAX];
    constexpr int KV = STEP == ET_CONTRACT ? ET_KMAX : 3;      // per-thread partials this step can produce
    const int r = blockIdx.y, K = et_k(STEP, P.n_p);
    double v[KV];
#pragma unroll
    for (int k = 0; k < KV; ++k) v[k] = 0.0;
    const int idx = blockIdx.x * ET_NT + threadIdx.x;
    if (act[r] && idx < nsites) et_site<STEP>(P, F, r, idx, coef ? coef[r] : 0.0f, v);
    if (K == 0) return;                                   // uniform over the block
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int k = 0; k < K; ++k) {
        double u = v[k];
        for (int o = 16; o > 0; o >>= 1) u += __shfl_down_sync(0xffffffffu, u, o);
        if (lane == 0) sh[warp][k] = u;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < K; k += ET_NT) {
        double s = 0.0;
        for (int w = 0; w < ET_NT / 32; ++w) s += sh[w][k];
        partials[((size_t)r * nblk + blockIdx.x) * K + k] = s;
    }
}

// totals[r K + k] = sum over the blocks of task r, in block order
__global__ void k_et_total(int R, int K, int nblk, const double *partials, double *totals) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < R * K; t += gridDim.x * blockDim.x) {
        const int r = t / K, k = t - r * K;
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += partials[((size_t)r * nblk + b) * K + k];
        totals[t] = s;
    }
}

// ---------------------------------------------------------------- executors
struct ETDev {
    pt_ctx *c = nullptr;
    ETP P;
    ETF F;
    int R = 0;
    int *d_act = nullptr;
    float *d_coef = nullptr;
    double *d_part = nullptr, *d_tot = nullptr;
    std::vector<void *> owned;
    void *get(size_t bytes) {
        void *p = nullptr;
        if (cudaMallocAsync(&p, bytes, c->stream) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        owned.push_back(p);
        return p;
    }
    ~ETDev() {
        for (void *p : owned) cudaFreeAsync(p, c->stream);
    }
    bool init() {   // fields and scratch for R tasks
        const size_t nh = (size_t)R * P.g.Nh;
        const int nblk = (P.g.N + ET_NT - 1) / ET_NT;
        F.x64 = (double *)get(nh * 8);
        F.t64 = (double *)get(nh * 8);
        F.r = (float *)get(nh * 4);
        F.p = (float *)get(nh * 4);
        F.q = (float *)get(nh * 4);
        F.e = (float *)get(nh * 4);
        F.t = (float *)get(nh * 4);
        d_act = (int *)get((size_t)R * 4);
        d_coef = (float *)get((size_t)R * 4);
        d_part = (double *)get((size_t)R * nblk * ET_KMAX * 8);
        d_tot = (double *)get((size_t)R * ET_KMAX * 8);
        for (void *p : owned)
            if (!p) return false;
        return cudaMemsetAsync(F.x64, 0, nh * 8, c->stream) == cudaSuccess;
    }
    template <int STEP>
    int step(const std::vector<int> &act, const std::vector<float> *coef, std::vector<double> *tot) {
        const int nsites = STEP == ET_CONTRACT ? P.g.N : P.g.Nh;
        const int nblk = (nsites + ET_NT - 1) / ET_NT, K = et_k(STEP, P.n_p);
        PT_CUDA(cudaMemcpyAsync(d_act, act.data(), (size_t)R * 4, cudaMemcpyHostToDevice, c->stream));
        if (coef) PT_CUDA(cudaMemcpyAsync(d_coef, coef->data(), (size_t)R * 4, cudaMemcpyHostToDevice, c->stream));
        k_et_step<STEP><<<dim3(nblk, R), ET_NT, 0, c->stream>>>(P, F, d_act, coef ? d_coef : nullptr, nsites, nblk,
                                                                d_part);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        if (K) {
            const int total = R * K;
            k_et_total<<<std::max(1, std::min((total + 255) / 256, 4 * c->num_sms)), 256, 0, c->stream>>>(
                R, K, nblk, d_part, d_tot);
            ++pt_kernel_launch_count;
            PT_CUDA(cudaGetLastError());
            tot->assign((size_t)R * K, 0.0);
            PT_CUDA(cudaMemcpyAsync(tot->data(), d_tot, (size_t)R * K * 8, cudaMemcpyDeviceToHost, c->stream));
            PT_CUDA(cudaStreamSynchronize(c->stream));      // the host needs the totals now
        }
        // (steps without a reduction return at once: an upload from pageable
        // memory is staged before cudaMemcpyAsync returns, so the host vectors may
        // change; such an upload also waits for the stream first, which pinned
        // staging buffers would avoid)
        return PT_OK;
    }
};

struct ETHost {
    pt_ctx *c = nullptr;          // unused on the host
    ETP P;
    ETF F;
    int R = 0;
    std::vector<double> x64, t64;
    std::vector<float> r, p, q, e, t;
    bool init() {
        const size_t nh = (size_t)R * P.g.Nh;
        x64.assign(nh, 0.0);
        t64.assign(nh, 0.0);
        r.assign(nh, 0.f);
        p.assign(nh, 0.f);
        q.assign(nh, 0.f);
        e.assign(nh, 0.f);
        t.assign(nh, 0.f);
        F = ETF{x64.data(), t64.data(), r.data(), p.data(), q.data(), e.data(), t.data()};
        return true;
    }
    template <int STEP>
    int step(const std::vector<int> &act, const std::vector<float> *coef, std::vector<double> *tot) {
        const int nsites = STEP == ET_CONTRACT ? P.g.N : P.g.Nh, K = et_k(STEP, P.n_p);
        if (K) tot->assign((size_t)R * K, 0.0);
        for (int rr = 0; rr < R; ++rr) {
            if (!act[rr]) continue;
            double v[ET_KMAX];
            for (int k = 0; k < ET_KMAX; ++k) v[k] = 0.0;
            for (int i = 0; i < nsites; ++i) et_site<STEP>(P, F, rr, i, coef ? (*coef)[rr] : 0.0f, v);
            for (int k = 0; k < K; ++k) (*tot)[(size_t)rr * K + k] = v[k];
        }
        return PT_OK;
    }
};

// ---------------------------------------------------------------- the batch
struct ETStats {
    int64_t inner = 0, outer = 0, kernel_steps = 0;
    double max_relres = 0.0;
    int noconv = 0;
};

// R tasks from x = 0 to the FP64 tolerance, then the contraction:
// out[(r n_p + n) 2 + {0, 1}] = q_n of task r
template <class X>
static int et_batch(X &ex, int R, double tol, int maxit, double delta, double *out, ETStats *S) {
    const ETP &P = ex.P;
    std::vector<int> act(R, 1), done(R, 0), on(R, 0), total(R, 0);
    std::vector<double> bn2(R, 0.0), rr(R, 0.0), target2(R, 0.0), tot;
    std::vector<float> beta(R, 0.0f), alpha(R, 0.0f);
    int rc;
    for (int outer = 0;; ++outer) {
        for (int r = 0; r < R; ++r) act[r] = !done[r];
        if ((rc = ex.template step<ET_OUTER1>(act, nullptr, nullptr)) ||
            (rc = ex.template step<ET_OUTER2>(act, nullptr, &tot)))
            return rc;
        S->kernel_steps += 2;
        bool any = false;
        for (int r = 0; r < R; ++r) {
            if (!act[r]) continue;
            const double r2 = tot[3 * r], b2 = tot[3 * r + 1], s2 = tot[3 * r + 2];
            if (outer == 0) bn2[r] = b2;
            if (!std::isfinite(r2) || !std::isfinite(s2)) {
                pt_set_error("even-odd trace: non-finite residual (task %d)", r);
                return PT_ERR_NUMERIC;
            }
            const double rel = bn2[r] > 0.0 ? sqrt(r2 / bn2[r]) : 0.0;
            S->outer += 1;
            const bool conv = bn2[r] == 0.0 || rel <= tol;
            if (conv || total[r] >= maxit) {
                done[r] = 1;
                S->max_relres = std::max(S->max_relres, rel);
                if (!conv) S->noconv += 1;
                continue;
            }
            any = true;
            on[r] = 1;
            rr[r] = s2;
            target2[r] = std::max(delta * delta * s2, 0.25 * tol * tol * bn2[r]);
            beta[r] = 0.0f;
        }
        if (!any) break;
        for (;;) {                                                   // inner CG from e = p = 0
            bool live = false;
            for (int r = 0; r < R; ++r) live = live || on[r];
            if (!live) break;
            if ((rc = ex.template step<ET_INNERA>(on, &beta, nullptr)) ||
                (rc = ex.template step<ET_INNERB>(on, &beta, &tot)))
                return rc;
            for (int r = 0; r < R; ++r) {
                alpha[r] = 0.0f;
                if (!on[r]) continue;
                if (!(tot[r] > 0.0)) { on[r] = 0; continue; }          // p = 0: nothing left to reduce
                alpha[r] = (float)(rr[r] / tot[r]);
            }
            if ((rc = ex.template step<ET_INNERC>(on, &alpha, &tot))) return rc;
            S->kernel_steps += 3;
            for (int r = 0; r < R; ++r) {
                if (!on[r]) continue;
                const double rn = tot[r];
                total[r] += 1;
                S->inner += 1;
                beta[r] = (float)(rn / rr[r]);
                rr[r] = rn;
                if (rn <= target2[r] || total[r] >= maxit) on[r] = 0;
            }
        }
        for (int r = 0; r < R; ++r) act[r] = !done[r];
        if ((rc = ex.template step<ET_UPDATE>(act, nullptr, nullptr))) return rc;   // x64 += e
        S->kernel_steps += 1;
    }
    std::fill(act.begin(), act.end(), 1);
    if ((rc = ex.template step<ET_CONTRACT>(act, nullptr, &tot))) return rc;
    S->kernel_steps += 1;
    for (size_t k = 0; k < (size_t)R * 2 * P.n_p; ++k) out[k] = tot[k];
    return PT_OK;
}

// all n_sets x m tasks in batches of at most Rmax; est_out[s][n] (complex)
// sums the colours' q_n of set s in colour order
template <class X>
static int et_run(X &ex, int n_tasks, int Rmax, double tol, int maxit, double delta, int n_sets, double *est_out,
                  ETStats *S) {
    const ETP P0 = ex.P;
    std::vector<double> q((size_t)n_tasks * 2 * P0.n_p, 0.0);
    for (int t0 = 0; t0 < n_tasks; t0 += Rmax) {
        const int R = std::min(Rmax, n_tasks - t0);
        X bx;
        bx.P = P0;
        bx.P.t0 = t0;
        bx.R = R;
        bx.c = ex.c;
        if (!bx.init()) {
            pt_set_error("even-odd trace: allocation of %d tasks' fields failed", R);
            return PT_ERR_OOM;
        }
        const int rc = et_batch(bx, R, tol, maxit, delta, q.data() + (size_t)t0 * 2 * P0.n_p, S);
        if (rc) return rc;
    }
    for (int s = 0; s < n_sets; ++s)
        for (int n = 0; n < P0.n_p; ++n) {
            double re = 0.0, im = 0.0;
            for (int c = 0; c < P0.m; ++c) {
                const size_t k = ((size_t)(s * P0.m + c) * P0.n_p + n) * 2;
                re += q[k];
                im += q[k + 1];
            }
            est_out[((size_t)s * P0.n_p + n) * 2] = re;
            est_out[((size_t)s * P0.n_p + n) * 2 + 1] = im;
        }
    return PT_OK;
}

// ---------------------------------------------------------------- entry points
static int et_params(const int dims[4], double m2, int n_colours, int mu, const int *p_list, int n_p, int noise,
                     uint64_t seed, int set0, int n_sets, double tol, int maxit, double delta, ETP *P,
                     const char *fn) {
    PT_CHECK_ARG(dims && p_list, "%s: NULL argument", fn);
    long N = 1;
    for (int k = 0; k < 4; ++k) {
        PT_CHECK_ARG(dims[k] >= 2 && dims[k] % 2 == 0, "%s: every lattice side must be even", fn);
        N *= dims[k];
    }
    PT_CHECK_ARG(N <= (1L << 30), "%s: lattice too large", fn);
    PT_CHECK_ARG(n_colours >= 1 && mu >= 0 && mu < 4 && n_p >= 1 && n_p <= PT_MAX_P, "%s: bad colours, mu or n_p",
                 fn);
    // the Laplacian is real: its probes are real Z2 vectors (a complex Z4 probe
    // would be solved through its real part and contracted with its conjugate,
    // an estimate of half the trace)
    PT_CHECK_ARG(noise == PT_NOISE_Z2, "%s: the real Laplacian takes Z2 noise", fn);
    PT_CHECK_ARG(set0 >= 0 && n_sets >= 1 && (long)n_sets * n_colours <= (1L << 30), "%s: bad sets", fn);
    PT_CHECK_ARG(tol > 0.0 && maxit >= 1 && delta > 0.0 && delta < 1.0, "%s: bad tol, maxit or delta", fn);
    P->g = make_eo_geom(dims);
    P->d = 8.0 + m2;
    P->seed = seed;
    P->noise = noise;
    P->mu = mu;
    P->n_p = n_p;
    P->m = n_colours;
    P->set0 = set0;
    P->t0 = 0;
    for (int k = 0; k < PT_MAX_P; ++k) P->p[k] = k < n_p ? p_list[k] : 0;
    return PT_OK;
}

static void et_fill_stats(pt_stats *st, const ETStats &S, int64_t n_tasks, int N, int Rmax, int64_t launches) {
    if (!st) return;
    *st = pt_stats{};
    st->n_rhs = n_tasks;
    st->inner_iters = S.inner;
    st->outer_iters = S.outer;
    st->site_rhs_applies = S.inner * (int64_t)N;      // one S apply = two half-lattice hops
    st->engine_iters = S.kernel_steps;
    st->kernel_launches = launches;
    st->max_relres = S.max_relres;
    st->n_slots = Rmax;
    st->n_noconv = S.noconv;
}

extern "C" int pt_trace_PAinv_eo(pt_ctx *c, const pt_op *op, const int32_t *col_dev, int n_colours, int mu,
                                 const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets,
                                 double tol, int maxit, double delta, double *est_out, pt_stats *stats) {
    PT_CHECK_ARG(c && op && op->ctx == c && op->kind == 0, "pt_trace_PAinv_eo: a Laplacian operator is required");
    PT_CHECK_ARG(col_dev && est_out, "pt_trace_PAinv_eo: NULL argument");
    ETDev ex;
    int rc = et_params(op->dims, op->m2, n_colours, mu, p_list, n_p, noise, seed, set0, n_sets, tol, maxit, delta,
                       &ex.P, "pt_trace_PAinv_eo");
    if (rc) return rc;
    PT_CUDA(cudaSetDevice(c->device));
    ex.c = c;
    ex.P.col = col_dev;
    const int64_t n_tasks = (int64_t)n_sets * n_colours;
    const size_t per_task = (size_t)ex.P.g.Nh * (2 * 8 + 5 * 4) +
                            (size_t)((ex.P.g.N + ET_NT - 1) / ET_NT) * ET_KMAX * 8 + ET_KMAX * 8 + 8;
    const size_t budget = c->mem_budget ? c->mem_budget : ((size_t)16 << 30);
    int Rmax = (int)std::min<int64_t>(n_tasks, std::max<int64_t>(1, (int64_t)(budget / per_task)));
    Rmax = std::min(Rmax, 65535);
    if (c->max_slots > 0) Rmax = std::min(Rmax, c->max_slots);
    ETStats S;
    const int64_t l0 = pt_kernel_launch_count;
    rc = et_run(ex, (int)n_tasks, Rmax, tol, maxit, delta, n_sets, est_out, &S);
    et_fill_stats(stats, S, n_tasks, ex.P.g.N, Rmax, pt_kernel_launch_count - l0);
    if (rc) return rc;
    if (S.noconv) {
        pt_set_error("pt_trace_PAinv_eo: %d right-hand sides did not converge", S.noconv);
        return PT_ERR_NOCONV;
    }
    return PT_OK;
}

extern "C" int pt_trace_PAinv_eo_host(const int dims[4], double m2, const int32_t *col_host, int n_colours, int mu,
                                      const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets,
                                      double tol, int maxit, double delta, double *est_out, pt_stats *stats) {
    PT_CHECK_ARG(col_host && est_out, "pt_trace_PAinv_eo_host: NULL argument");
    ETHost ex;
    int rc = et_params(dims, m2, n_colours, mu, p_list, n_p, noise, seed, set0, n_sets, tol, maxit, delta, &ex.P,
                       "pt_trace_PAinv_eo_host");
    if (rc) return rc;
    ex.P.col = col_host;
    const int64_t n_tasks = (int64_t)n_sets * n_colours;
    ETStats S;
    rc = et_run(ex, (int)n_tasks, (int)n_tasks, tol, maxit, delta, n_sets, est_out, &S);
    et_fill_stats(stats, S, n_tasks, ex.P.g.N, (int)n_tasks, 0);
    if (rc) return rc;
    if (S.noconv) {
        pt_set_error("pt_trace_PAinv_eo_host: %d right-hand sides did not converge", S.noconv);
        return PT_ERR_NOCONV;
    }
    return PT_OK;
}
