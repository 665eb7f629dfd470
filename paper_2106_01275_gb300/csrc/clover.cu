// Clover (Sheikholeslami-Wohlert) site blocks of the Wilson-Dirac operator,
// their application and their inverses (the operator-fidelity step after
// deflation; the paper's production operator is a clover Wilson matrix,
// Sec. 4.2, which it takes from the lattice literature).
//
//   (A_c psi)(x) = (A_W psi)(x) + C(x) psi(x),
//   C(x) = -kappa c_sw sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x),
//   sigma_{mu nu} = (i/2) [g_mu, g_nu],   F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^H) / (8 i),
// Q_{mu nu}(x) the sum of the four plaquettes in the (mu, nu) plane that start
// and end at x, each run the same way round.  The gamma matrices are the
// chiral basis of the library's hopping term.
//
// The per-site arithmetic is in __host__ __device__ functions: the device
// kernels and the host-only entry points (which tests run without a GPU) call
// the same code.
#include <algorithm>

#include "hd_complex.cuh"
#include "pt_common.cuh"

// sigma_{mu nu} for the six planes mu < nu, in the order (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
struct SigmaTab {
    zd s[6][16];
};

static SigmaTab make_sigma() {
    SigmaTab T;
    int pl = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++pl) {
            zd gm[16], gn[16];
            gamma_chiral(mu, gm);
            gamma_chiral(nu, gn);
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j) {
                    zd c = {0.0, 0.0};
                    for (int k = 0; k < 4; ++k)
                        c = zadd(c, zsub(zmulc(gm[i * 4 + k], gn[k * 4 + j]), zmulc(gn[i * 4 + k], gm[k * 4 + j])));
                    T.s[pl][i * 4 + j] = {-0.5 * c.im, 0.5 * c.re};   // (i/2) c
                }
        }
    return T;
}

struct CloverGeom {
    int D[4];
    int stride[4];
    int N;
};

__host__ __device__ __forceinline__ int cl_step(const CloverGeom &g, int i, int mu, int s) {
    const int x = (i / g.stride[mu]) % g.D[mu];
    if (s > 0) return (x == g.D[mu] - 1) ? i - (g.D[mu] - 1) * g.stride[mu] : i + g.stride[mu];
    return (x == 0) ? i + (g.D[mu] - 1) * g.stride[mu] : i - g.stride[mu];
}

// 3 x 3 products of links taken forward (U) or backward (U^H)
template <class L>
__host__ __device__ __forceinline__ void cl_link(const L &U, int site, int mu, bool dag, zd m[9]) {
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) m[a * 3 + b] = dag ? zconj(U(site, mu, b * 3 + a)) : U(site, mu, a * 3 + b);
}
__host__ __device__ __forceinline__ void cl_mul(const zd a[9], const zd b[9], zd c[9]) {
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            zd t = {0.0, 0.0};
            for (int k = 0; k < 3; ++k) t = zadd(t, zmulc(a[i * 3 + k], b[k * 3 + j]));
            c[i * 3 + j] = t;
        }
}

// transporter around a closed path of four steps from site i: step (mu, +1)
// multiplies by U_mu(y), step (mu, -1) by U_mu(y - mu)^H
template <class L>
__host__ __device__ __forceinline__ void cl_loop(const L &U, const CloverGeom &g, int i, const int dirs[4],
                                                 const int sgn[4], zd out[9]) {
    zd M[9], l[9], t[9];
    for (int e = 0; e < 9; ++e) M[e] = {e % 4 == 0 ? 1.0 : 0.0, 0.0};
    int y = i;
    for (int s = 0; s < 4; ++s) {
        if (sgn[s] > 0) {
            cl_link(U, y, dirs[s], false, l);
            y = cl_step(g, y, dirs[s], 1);
        } else {
            y = cl_step(g, y, dirs[s], -1);
            cl_link(U, y, dirs[s], true, l);
        }
        cl_mul(M, l, t);
        for (int e = 0; e < 9; ++e) M[e] = t[e];
    }
    for (int e = 0; e < 9; ++e) out[e] = M[e];
}

// C(x) at site i as 12 x 12 complex, row-major, component = 3 spin + colour
template <class L>
__host__ __device__ void clover_site(const L &U, const CloverGeom &g, const SigmaTab &S, int i, double kappa,
                                     double csw, zd C[144]) {
    for (int e = 0; e < 144; ++e) C[e] = {0.0, 0.0};
    int pl = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++pl) {
            zd Q[9], P[9];
            for (int e = 0; e < 9; ++e) Q[e] = {0.0, 0.0};
            const int d1[4] = {mu, nu, mu, nu}, s1[4] = {1, 1, -1, -1};
            const int d2[4] = {nu, mu, nu, mu}, s2[4] = {1, -1, -1, 1};
            const int d3[4] = {mu, nu, mu, nu}, s3[4] = {-1, -1, 1, 1};
            const int d4[4] = {nu, mu, nu, mu}, s4[4] = {-1, 1, 1, -1};
            cl_loop(U, g, i, d1, s1, P);
            for (int e = 0; e < 9; ++e) Q[e] = zadd(Q[e], P[e]);
            cl_loop(U, g, i, d2, s2, P);
            for (int e = 0; e < 9; ++e) Q[e] = zadd(Q[e], P[e]);
            cl_loop(U, g, i, d3, s3, P);
            for (int e = 0; e < 9; ++e) Q[e] = zadd(Q[e], P[e]);
            cl_loop(U, g, i, d4, s4, P);
            for (int e = 0; e < 9; ++e) Q[e] = zadd(Q[e], P[e]);
            // F = (Q - Q^H) / (8 i): with D = Q - Q^H, D / (8 i) = (Im D, -Re D) / 8
            zd F[9];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const zd d = zsub(Q[a * 3 + b], zconj(Q[b * 3 + a]));
                    F[a * 3 + b] = {d.im / 8.0, -d.re / 8.0};
                }
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t) {
                    const zd sg = S.s[pl][s * 4 + t];
                    if (sg.re == 0.0 && sg.im == 0.0) continue;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) {
                            zd &c = C[(s * 3 + a) * 12 + t * 3 + b];
                            c = zadd(c, zmulc(sg, F[a * 3 + b]));
                        }
                }
        }
    const double f = -kappa * csw;
    for (int e = 0; e < 144; ++e) C[e] = zscal(C[e], f);
}

// inverse of a 12 x 12 complex matrix by Gauss-Jordan elimination with
// partial pivoting (row swaps); returns false if a pivot vanishes
__host__ __device__ bool inv12(const zd A[144], zd X[144]) {
    zd M[144];
    for (int e = 0; e < 144; ++e) { M[e] = A[e]; X[e] = {e % 13 == 0 ? 1.0 : 0.0, 0.0}; }
    for (int col = 0; col < 12; ++col) {
        int piv = col;
        double best = M[col * 12 + col].re * M[col * 12 + col].re + M[col * 12 + col].im * M[col * 12 + col].im;
        for (int r = col + 1; r < 12; ++r) {
            const zd v = M[r * 12 + col];
            const double n = v.re * v.re + v.im * v.im;
            if (n > best) { best = n; piv = r; }
        }
        if (!(best > 0.0)) return false;
        if (piv != col)
            for (int k = 0; k < 12; ++k) {
                zd t = M[col * 12 + k]; M[col * 12 + k] = M[piv * 12 + k]; M[piv * 12 + k] = t;
                t = X[col * 12 + k]; X[col * 12 + k] = X[piv * 12 + k]; X[piv * 12 + k] = t;
            }
        const zd p = M[col * 12 + col];
        const zd pinv = {p.re / best, -p.im / best};                     // 1 / p
        for (int k = 0; k < 12; ++k) { M[col * 12 + k] = zmulc(M[col * 12 + k], pinv); X[col * 12 + k] = zmulc(X[col * 12 + k], pinv); }
        for (int r = 0; r < 12; ++r) {
            if (r == col) continue;
            const zd f = M[r * 12 + col];
            if (f.re == 0.0 && f.im == 0.0) continue;
            for (int k = 0; k < 12; ++k) {
                M[r * 12 + k] = zsub(M[r * 12 + k], zmulc(f, M[col * 12 + k]));
                X[r * 12 + k] = zsub(X[r * 12 + k], zmulc(f, X[col * 12 + k]));
            }
        }
    }
    return true;
}

// ---------------------------------------------------------------- kernels
__global__ void k_clover_blocks(CloverGeom g, SigmaTab S, PackedLinks U, double kappa, double csw, double *out) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < g.N; i += gridDim.x * blockDim.x) {
        zd C[144];
        clover_site(U, g, S, i, kappa, csw, C);
        double *o = out + (size_t)i * 288;
        for (int e = 0; e < 144; ++e) { o[2 * e] = C[e].re; o[2 * e + 1] = C[e].im; }
    }
}

// y[r][i] = beta y[r][i] + B(i) x[r][i] per site (B: [N][12][12] complex)
__global__ void k_site_blocks_apply(int N, const double *B, const double *x, double beta, int nrhs, double *y) {
    const long total = (long)nrhs * N;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int i = (int)(t % N);
        const double *b = B + (size_t)i * 288, *xv = x + (size_t)t * 24;
        double *yv = y + (size_t)t * 24;
        zd xs[12];
        for (int c = 0; c < 12; ++c) xs[c] = {xv[2 * c], xv[2 * c + 1]};
        for (int r = 0; r < 12; ++r) {
            zd acc = {0.0, 0.0};
            for (int c = 0; c < 12; ++c) acc = zadd(acc, zmulc({b[(r * 12 + c) * 2], b[(r * 12 + c) * 2 + 1]}, xs[c]));
            if (beta != 0.0) acc = zadd(acc, zscal({yv[2 * r], yv[2 * r + 1]}, beta));
            yv[2 * r] = acc.re;
            yv[2 * r + 1] = acc.im;
        }
    }
}

// Binv(i) = (shift 1 + B(i))^{-1}; bad[0] counts singular blocks
__global__ void k_site_blocks_invert(int N, const double *B, double shift, double *Binv, int *bad) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
        zd A[144], X[144];
        const double *b = B + (size_t)i * 288;
        for (int e = 0; e < 144; ++e) A[e] = {b[2 * e] + (e % 13 == 0 ? shift : 0.0), b[2 * e + 1]};
        if (!inv12(A, X)) atomicAdd(bad, 1);
        double *o = Binv + (size_t)i * 288;
        for (int e = 0; e < 144; ++e) { o[2 * e] = X[e].re; o[2 * e + 1] = X[e].im; }
    }
}

// ---------------------------------------------------------------- host side
static int clover_geom(const int dims[4], CloverGeom *g) {
    long N = 1;
    for (int mu = 0; mu < 4; ++mu) {
        PT_CHECK_ARG(dims[mu] >= 1, "clover: lattice sides must be positive");
        g->D[mu] = dims[mu];
        g->stride[mu] = (int)N;
        N *= dims[mu];
    }
    PT_CHECK_ARG(N <= (1L << 30), "clover: lattice too large");
    g->N = (int)N;
    return PT_OK;
}

extern "C" int pt_clover_blocks_host(const int dims[4], const double *U_host, double kappa, double csw,
                                     double *blocks_out) {
    PT_CHECK_ARG(dims && U_host && blocks_out, "pt_clover_blocks_host: NULL argument");
    CloverGeom g;
    int rc = clover_geom(dims, &g);
    if (rc) return rc;
    const SigmaTab S = make_sigma();
    const UserLinks U{U_host};
    for (int i = 0; i < g.N; ++i) {
        zd C[144];
        clover_site(U, g, S, i, kappa, csw, C);
        for (int e = 0; e < 144; ++e) {
            blocks_out[(size_t)i * 288 + 2 * e] = C[e].re;
            blocks_out[(size_t)i * 288 + 2 * e + 1] = C[e].im;
        }
    }
    return PT_OK;
}

extern "C" int pt_site_blocks_invert_host(int n, const double *blocks, double shift, double *inv_out) {
    PT_CHECK_ARG(n >= 0 && blocks && inv_out, "pt_site_blocks_invert_host: bad argument");
    for (int i = 0; i < n; ++i) {
        zd A[144], X[144];
        for (int e = 0; e < 144; ++e)
            A[e] = {blocks[(size_t)i * 288 + 2 * e] + (e % 13 == 0 ? shift : 0.0), blocks[(size_t)i * 288 + 2 * e + 1]};
        if (!inv12(A, X)) {
            pt_set_error("pt_site_blocks_invert_host: block %d is singular", i);
            return PT_ERR_NUMERIC;
        }
        for (int e = 0; e < 144; ++e) {
            inv_out[(size_t)i * 288 + 2 * e] = X[e].re;
            inv_out[(size_t)i * 288 + 2 * e + 1] = X[e].im;
        }
    }
    return PT_OK;
}

extern "C" int pt_clover_blocks(pt_ctx *c, const pt_op *op, double csw, double *blocks_dev) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_clover_blocks: bad context/operator");
    PT_CHECK_ARG(op->kind == 1, "pt_clover_blocks: a Wilson-Dirac operator is required");
    PT_CHECK_ARG(blocks_dev, "pt_clover_blocks: NULL output");
    PT_CUDA(cudaSetDevice(c->device));
    CloverGeom g;
    int rc = clover_geom(op->dims, &g);
    if (rc) return rc;
    const int grid = std::max(1, std::min((g.N + 127) / 128, 16 * c->num_sms));
    k_clover_blocks<<<grid, 128, 0, c->stream>>>(g, make_sigma(), PackedLinks{op->U64, g.N}, op->kappa, csw,
                                                 blocks_dev);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}

extern "C" int pt_site_blocks_apply(pt_ctx *c, int N, const double *blocks_dev, const double *x_dev, double beta,
                                    double *y_dev, int nrhs) {
    PT_CHECK_ARG(c && N >= 1 && nrhs >= 0 && nrhs <= 65535, "pt_site_blocks_apply: bad argument");
    if (nrhs == 0) return PT_OK;
    PT_CHECK_ARG(blocks_dev && x_dev && y_dev && x_dev != (const double *)y_dev,
                 "pt_site_blocks_apply: NULL or aliased fields");
    PT_CUDA(cudaSetDevice(c->device));
    const long total = (long)nrhs * N;
    const int grid = (int)std::max(1L, std::min((total + 127) / 128, 64L * c->num_sms));
    k_site_blocks_apply<<<grid, 128, 0, c->stream>>>(N, blocks_dev, x_dev, beta, nrhs, y_dev);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}

extern "C" int pt_site_blocks_invert(pt_ctx *c, int N, const double *blocks_dev, double shift, double *inv_dev) {
    PT_CHECK_ARG(c && N >= 1 && blocks_dev && inv_dev && (const double *)inv_dev != blocks_dev,
                 "pt_site_blocks_invert: bad argument");
    PT_CUDA(cudaSetDevice(c->device));
    int *bad = nullptr;
    if (cudaMallocAsync((void **)&bad, sizeof(int), c->stream) != cudaSuccess) {
        cudaGetLastError();
        pt_set_error("pt_site_blocks_invert: device allocation failed");
        return PT_ERR_OOM;
    }
    int rc = PT_OK, h_bad = 0;
    do {
        if (cudaMemsetAsync(bad, 0, sizeof(int), c->stream) != cudaSuccess) {
            rc = pt_cuda_fail(cudaGetLastError(), "cudaMemsetAsync", __FILE__, __LINE__);
            break;
        }
        const int grid = std::max(1, std::min((N + 127) / 128, 16 * c->num_sms));
        k_site_blocks_invert<<<grid, 128, 0, c->stream>>>(N, blocks_dev, shift, inv_dev, bad);
        ++pt_kernel_launch_count;
        cudaError_t ce = cudaGetLastError();
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
        if (ce != cudaSuccess) { rc = pt_cuda_fail(ce, "k_site_blocks_invert", __FILE__, __LINE__); break; }
        if (h_bad) {
            pt_set_error("pt_site_blocks_invert: %d singular blocks", h_bad);
            rc = PT_ERR_NUMERIC;
        }
    } while (0);
    cudaFreeAsync(bad, c->stream);
    return rc;
}
