// Deflation of given singular triplets (Sec. 2.4, Eq. (6)) for the displaced
// trace.  With U, V (n_ev columns) and M = (U^H A V)^{-1}:
//   Tr(P A^{-1}) = Tr(M U^H P V) + Tr(P A^{-1} (I - Q)),
// and a probe v contributes v^H P A^{-1} v - (v^H P V) M (U^H v) to the
// second part.  The probe contractions with A^{-1} come from the solver
// engine (pt_trace_PAinv_multi); this file computes what needs no solve: the
// Gram matrices U^H P_n V and, per probe, v^H P_n V and U^H v.
#include <vector>

#include "pt_common.cuh"

#define PT_DEFL_MAXP 16

struct DeflArgs {
    int p[PT_DEFL_MAXP];
};

// K2 doubles per thread summed over the CTA in a fixed order; thread 0 writes them
template <int K2>
__device__ __forceinline__ void defl_block_sum(double (&v)[K2], double *sh, double *out, int k_used) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int k = 0; k < K2; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
    __syncthreads();
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K2; ++k) sh[warp * K2 + k] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
        for (int k = 0; k < k_used; ++k) {
            double s = 0.0;
            for (int w = 0; w < nw; ++w) s += sh[w * K2 + k];
            out[k] = s;
        }
}

// one CTA per (probe t, triplet i): over the sites of the probe's colour,
//   beta_i = U_i^H v = sum conj(U_i(x, a)) z(x),
//   alpha_{n,i} = v^H P_n V_i = sum conj(z(x)) V_i(x + p_n e_mu, a).
// out[t][i][n] = alpha_{n,i} (n < n_p), out[t][i][n_p] = beta_i, complex.
__global__ void __launch_bounds__(256) k_defl_probe_dots(Geom g, int dof, const int32_t *__restrict__ col,
                                                         const int4 *__restrict__ task, int n_tasks, int n_ev,
                                                         const double2 *__restrict__ U, const double2 *__restrict__ V,
                                                         uint64_t seed, int noise, int mu, int n_p, DeflArgs A,
                                                         double *out) {
    __shared__ double sh[32 * 2 * (PT_DEFL_MAXP + 1)];
    const int N = g.N;
    for (long b = blockIdx.x; b < (long)n_tasks * n_ev; b += gridDim.x) {
        const int t = (int)(b / n_ev), i = (int)(b % n_ev);
        const int4 tk = task[t];                           // (set, colour, component, -)
        const uint64_t key = pt_set_key(seed, tk.x);
        double acc[2 * (PT_DEFL_MAXP + 1)];
#pragma unroll
        for (int k = 0; k < 2 * (PT_DEFL_MAXP + 1); ++k) acc[k] = 0.0;
        for (int x = threadIdx.x; x < N; x += blockDim.x) {
            if (col[x] != tk.y) continue;
            int xc[4];
            site_coords(g, x, xc);
            const Cx<double> z = pt_noise(key, (uint64_t)x, noise);
            const double2 u = U[((size_t)i * N + x) * dof + tk.z];
            const Cx<double> be = cconjmul(Cx<double>{u.x, u.y}, z);
            acc[2 * n_p] += be.re;
            acc[2 * n_p + 1] += be.im;
#pragma unroll
            for (int n = 0; n < PT_DEFL_MAXP; ++n) {
                if (n >= n_p) break;
                const int y = shift_site(g, x, xc, mu, A.p[n]);
                const double2 w = V[((size_t)i * N + y) * dof + tk.z];
                const Cx<double> al = cconjmul(z, Cx<double>{w.x, w.y});
                acc[2 * n] += al.re;
                acc[2 * n + 1] += al.im;
            }
        }
        defl_block_sum<2 * (PT_DEFL_MAXP + 1)>(acc, sh, out + b * 2 * (n_p + 1), 2 * (n_p + 1));
        __syncthreads();
    }
}

// one CTA per (n, i, j): G[n][i][j] = (U^H P_n V)_ij = sum_{x,a} conj(U_i(x, a)) V_j(x + p_n e_mu, a)
__global__ void __launch_bounds__(256) k_defl_gram(Geom g, int dof, int n_ev, const double2 *__restrict__ U,
                                                   const double2 *__restrict__ V, int mu, int n_p, DeflArgs A,
                                                   double *G) {
    __shared__ double sh[32 * 2];
    const int N = g.N;
    for (long b = blockIdx.x; b < (long)n_p * n_ev * n_ev; b += gridDim.x) {
        const int n = (int)(b / ((long)n_ev * n_ev)), i = (int)((b / n_ev) % n_ev), j = (int)(b % n_ev);
        double acc[2] = {0.0, 0.0};
        for (int x = threadIdx.x; x < N; x += blockDim.x) {
            int xc[4];
            site_coords(g, x, xc);
            const int y = shift_site(g, x, xc, mu, A.p[n]);
            for (int a = 0; a < dof; ++a) {
                const double2 u = U[((size_t)i * N + x) * dof + a], w = V[((size_t)j * N + y) * dof + a];
                const Cx<double> q = cconjmul(Cx<double>{u.x, u.y}, Cx<double>{w.x, w.y});
                acc[0] += q.re;
                acc[1] += q.im;
            }
        }
        defl_block_sum<2>(acc, sh, G + b * 2, 2);
        __syncthreads();
    }
}

extern "C" int pt_deflation_terms(pt_ctx *c, const pt_op *op, const int32_t *col_dev, int n_colours, int mu,
                                  const int *p_list, int n_p, int noise, uint64_t seed, int set0, int n_sets,
                                  int n_ev, const double *U_dev, const double *V_dev, const double *M_host,
                                  double *corr_out, double *exact_out) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_deflation_terms: bad context/operator");
    PT_CHECK_ARG(col_dev && p_list && U_dev && V_dev && M_host && corr_out && exact_out,
                 "pt_deflation_terms: NULL argument");
    PT_CHECK_ARG(n_colours >= 1 && n_sets >= 1 && set0 >= 0 && mu >= 0 && mu < 4, "pt_deflation_terms: bad sizes");
    PT_CHECK_ARG(n_p >= 1 && n_p <= PT_DEFL_MAXP, "pt_deflation_terms: 1 <= n_p <= %d", PT_DEFL_MAXP);
    PT_CHECK_ARG(n_ev >= 1 && n_ev <= 4096, "pt_deflation_terms: 1 <= n_ev <= 4096");
    PT_CHECK_ARG(noise == PT_NOISE_Z2 || (noise == PT_NOISE_Z4 && op->dof == 12),
                 "pt_deflation_terms: Z4 noise needs the complex (Wilson) operator");
    PT_CUDA(cudaSetDevice(c->device));
    const int dof = op->dof;
    const Geom g = op->g;
    std::vector<int4> tasks;
    for (int s = 0; s < n_sets; ++s)
        for (int col = 0; col < n_colours; ++col)
            for (int a = 0; a < dof; ++a) tasks.push_back(make_int4(set0 + s, col, a, 0));
    const int n_tasks = (int)tasks.size();
    DeflArgs A;
    for (int n = 0; n < PT_DEFL_MAXP; ++n) A.p[n] = n < n_p ? p_list[n] : 0;
    const size_t dots_n = (size_t)n_tasks * n_ev * (n_p + 1) * 2, gram_n = (size_t)n_p * n_ev * n_ev * 2;
    int4 *d_task = nullptr;
    double *d_dots = nullptr, *d_gram = nullptr;
    PT_CUDA(cudaMallocAsync((void **)&d_task, tasks.size() * sizeof(int4), c->stream));
    PT_CUDA(cudaMallocAsync((void **)&d_dots, dots_n * sizeof(double), c->stream));
    PT_CUDA(cudaMallocAsync((void **)&d_gram, gram_n * sizeof(double), c->stream));
    PT_CUDA(cudaMemcpyAsync(d_task, tasks.data(), tasks.size() * sizeof(int4), cudaMemcpyHostToDevice, c->stream));
    const int grid = 16 * c->num_sms;
    k_defl_probe_dots<<<grid, 256, 0, c->stream>>>(g, dof, col_dev, d_task, n_tasks, n_ev, (const double2 *)U_dev,
                                                   (const double2 *)V_dev, seed, noise, mu, n_p, A, d_dots);
    k_defl_gram<<<grid, 256, 0, c->stream>>>(g, dof, n_ev, (const double2 *)U_dev, (const double2 *)V_dev, mu, n_p, A,
                                             d_gram);
    pt_kernel_launch_count += 2;
    PT_CUDA(cudaGetLastError());
    std::vector<double> dots(dots_n), gram(gram_n);
    PT_CUDA(cudaMemcpyAsync(dots.data(), d_dots, dots_n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaMemcpyAsync(gram.data(), d_gram, gram_n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PT_CUDA(cudaFreeAsync(d_task, c->stream));
    PT_CUDA(cudaFreeAsync(d_dots, c->stream));
    PT_CUDA(cudaFreeAsync(d_gram, c->stream));
    PT_CUDA(cudaStreamSynchronize(c->stream));
    // the small contractions, in a fixed order: corr[s][n] += alpha_n^T M beta, exact[n] = sum M_ij G[n][j][i]
    auto Mij = [&](int i, int j) { return std::make_pair(M_host[(i * n_ev + j) * 2], M_host[(i * n_ev + j) * 2 + 1]); };
    for (size_t k = 0; k < (size_t)n_sets * n_p * 2; ++k) corr_out[k] = 0.0;
    std::vector<double> mb((size_t)n_ev * 2);
    for (int t = 0; t < n_tasks; ++t) {
        const double *d = dots.data() + (size_t)t * n_ev * (n_p + 1) * 2;
        for (int i = 0; i < n_ev; ++i) {       // (M beta)_i
            double re = 0.0, im = 0.0;
            for (int j = 0; j < n_ev; ++j) {
                const auto m = Mij(i, j);
                const double br = d[((size_t)j * (n_p + 1) + n_p) * 2], bi = d[((size_t)j * (n_p + 1) + n_p) * 2 + 1];
                re += m.first * br - m.second * bi;
                im += m.first * bi + m.second * br;
            }
            mb[2 * i] = re;
            mb[2 * i + 1] = im;
        }
        const int s = tasks[t].x - set0;
        for (int n = 0; n < n_p; ++n) {
            double re = 0.0, im = 0.0;
            for (int i = 0; i < n_ev; ++i) {
                const double ar = d[((size_t)i * (n_p + 1) + n) * 2], ai = d[((size_t)i * (n_p + 1) + n) * 2 + 1];
                re += ar * mb[2 * i] - ai * mb[2 * i + 1];
                im += ar * mb[2 * i + 1] + ai * mb[2 * i];
            }
            corr_out[((size_t)s * n_p + n) * 2] += re;
            corr_out[((size_t)s * n_p + n) * 2 + 1] += im;
        }
    }
    for (int n = 0; n < n_p; ++n) {
        double re = 0.0, im = 0.0;
        for (int i = 0; i < n_ev; ++i)
            for (int j = 0; j < n_ev; ++j) {
                const auto m = Mij(i, j);
                const double gr = gram[(((size_t)n * n_ev + j) * n_ev + i) * 2];
                const double gi = gram[(((size_t)n * n_ev + j) * n_ev + i) * 2 + 1];
                re += m.first * gr - m.second * gi;
                im += m.first * gi + m.second * gr;
            }
        exact_out[2 * n] = re;
        exact_out[2 * n + 1] = im;
    }
    return PT_OK;
}
