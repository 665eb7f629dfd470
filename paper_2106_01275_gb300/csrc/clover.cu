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
#include <cmath>

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

// ---------------------------------------------------------------- clover term of the batched engine
// 1 + C(x) commutes with g5 = diag(1, 1, -1, -1) (sigma_{mu nu} does) and is
// Hermitian (sigma_{mu nu} and F_{mu nu} are), so in the chiral basis it is
// two Hermitian 6 x 6 blocks, components 6q .. 6q + 5 for chirality q; so is
// its inverse.  Each block is packed as 36 reals: the six real diagonal
// entries, then the upper entries u_ij (i < j, row-major) as re, im.  Half
// entry h of parity par is the site 2h + b, b fixing the parity (D_0 even).
// Arrays, chunk-major by half entry: CL64 double2 [3][36][N/2] (1 + C on
// the even sites, (1 + C)^{-1} on the odd ones, 1 + C on the odd ones),
// CL32 float4 [2][18][N/2] (the first two).  bad counts blocks that are not
// of that form (an entry outside the chiral blocks, or an asymmetry, above
// 1e-9 of the block's largest entry).
__global__ void k_clover_pack(CloverGeom g, const double *C, const double *Cinv, double2 *CL64, float4 *CL32,
                              int *bad) {
    const int Nh = g.N / 2;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < 3 * Nh; t += gridDim.x * blockDim.x) {
        const int a = t / Nh, h = t - a * Nh;
        const int par = a == 0 ? 0 : 1;
        int r = 2 * h, ysum = 0;
        r /= g.D[0];
        for (int mu = 1; mu < 4; ++mu) {
            ysum += r % g.D[mu];
            r /= g.D[mu];
        }
        const int s = 2 * h + ((par ^ ysum) & 1);       // x_0 parity that gives the site parity par
        const double *M = (a == 1 ? Cinv : C) + (size_t)s * 288;
        auto ent = [&](int i, int j, double &re, double &im) {
            re = M[(i * 12 + j) * 2] + (a != 1 && i == j ? 1.0 : 0.0);
            im = M[(i * 12 + j) * 2 + 1];
        };
        double big = 0.0;
        for (int e = 0; e < 144; ++e) big = fmax(big, fabs(M[2 * e]) + fabs(M[2 * e + 1]));
        big = fmax(big, 1.0);
        bool ok = true;
        double w[72];
        for (int q = 0; q < 2; ++q) {
            double *wq = w + 36 * q;
            int k = 6;
            for (int i = 0; i < 6; ++i) {
                double re, im;
                ent(6 * q + i, 6 * q + i, re, im);
                wq[i] = re;
                ok = ok && fabs(im) <= 1e-9 * big;
                for (int j = 0; j < 6; ++j) {          // the other chirality's columns vanish
                    double ore, oim;
                    ent(6 * q + i, 6 * (1 - q) + j, ore, oim);
                    ok = ok && fabs(ore) + fabs(oim) <= 1e-9 * big;
                }
                for (int j = i + 1; j < 6; ++j) {
                    double ure, uim, lre, lim;
                    ent(6 * q + i, 6 * q + j, ure, uim);
                    ent(6 * q + j, 6 * q + i, lre, lim);
                    ok = ok && fabs(ure - lre) + fabs(uim + lim) <= 1e-9 * big;
                    wq[k] = ure;
                    wq[k + 1] = uim;
                    k += 2;
                }
            }
        }
        if (!ok) atomicAdd(bad, 1);
        for (int k = 0; k < 36; ++k) CL64[((size_t)a * 36 + k) * Nh + h] = make_double2(w[2 * k], w[2 * k + 1]);
        if (a < 2)
            for (int k = 0; k < 18; ++k)
                CL32[((size_t)a * 18 + k) * Nh + h] =
                    make_float4((float)w[4 * k], (float)w[4 * k + 1], (float)w[4 * k + 2], (float)w[4 * k + 3]);
    }
}

extern "C" int pt_op_set_clover(pt_op *op, double csw) {
    PT_CHECK_ARG(op && op->kind == 1, "pt_op_set_clover: a Wilson-Dirac operator is required");
    PT_CHECK_ARG(std::isfinite(csw), "pt_op_set_clover: c_sw must be finite");
    pt_ctx *c = op->ctx;
    PT_CUDA(cudaSetDevice(op->device));
    if (csw == 0.0) {
        PT_CUDA(cudaStreamSynchronize(c->stream));
        cudaFree(op->CL64);
        cudaFree(op->CL32);
        op->CL64 = nullptr;
        op->CL32 = nullptr;
        op->csw = 0.0;
        return PT_OK;
    }
    for (int mu = 0; mu < 4; ++mu)
        PT_CHECK_ARG(op->dims[mu] >= 2 && op->dims[mu] % 2 == 0,
                     "pt_op_set_clover: the clover operator runs on the even-odd engine: every side must be even");
    CloverGeom g;
    int rc = clover_geom(op->dims, &g);
    if (rc) return rc;
    const size_t Nh = (size_t)g.N / 2, nb = (size_t)g.N * 288 * sizeof(double);
    double *C = nullptr, *Cinv = nullptr;
    double2 *CL64 = nullptr;
    float4 *CL32 = nullptr;
    int *bad = nullptr;
    cudaError_t e = cudaMalloc((void **)&C, nb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&Cinv, nb);
    if (e == cudaSuccess) e = cudaMalloc((void **)&CL64, Nh * 3 * 36 * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc((void **)&CL32, Nh * 2 * 18 * sizeof(float4));
    if (e == cudaSuccess) e = cudaMalloc((void **)&bad, sizeof(int));
    auto release = [&](bool keep) {
        cudaFree(C);
        cudaFree(Cinv);
        cudaFree(bad);
        if (!keep) {
            cudaFree(CL64);
            cudaFree(CL32);
        }
    };
    if (e != cudaSuccess) {
        cudaGetLastError();
        release(false);
        pt_set_error("pt_op_set_clover: device allocation failed (%s)", cudaGetErrorString(e));
        return PT_ERR_OOM;
    }
    rc = pt_clover_blocks(c, op, csw, C);
    if (rc == PT_OK) rc = pt_site_blocks_invert(c, g.N, C, 1.0, Cinv);      // synchronises
    int h_bad = 0;
    if (rc == PT_OK) {
        e = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
        const int grid = std::max(1, std::min((int)((3 * Nh + 127) / 128), 16 * c->num_sms));
        if (e == cudaSuccess) {
            k_clover_pack<<<grid, 128, 0, c->stream>>>(g, C, Cinv, CL64, CL32, bad);
            ++pt_kernel_launch_count;
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) rc = pt_cuda_fail(e, "k_clover_pack", __FILE__, __LINE__);
        else if (h_bad) {
            pt_set_error("pt_op_set_clover: %d site blocks are not Hermitian chiral blocks", h_bad);
            rc = PT_ERR_NUMERIC;
        }
    }
    if (rc != PT_OK) {
        release(false);
        return rc;
    }
    release(true);
    cudaFree(op->CL64);
    cudaFree(op->CL32);
    op->CL64 = (double *)CL64;
    op->CL32 = (float *)CL32;
    op->csw = csw;
    return PT_OK;
}
