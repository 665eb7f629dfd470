// Even-odd (red-black) preconditioning of both operators, as building blocks.
//
// On a torus with every side even, each hop joins sites of opposite parity,
// so with the even sites first
//   A = [[A_ee, A_eo], [A_oe, A_oo]],  A_ee = A_oo = d I,
// d = 8 + m^2 and A_eo = -H_eo for the Laplacian (H the sum of the eight
// hops), d = 1 and A_eo = -kappa D_eo for Wilson (D the hopping term), and
// A x = b is solved through the Schur complement on the even sites:
//   S x_e = b'_e,  S = A_ee - A_eo A_oo^{-1} A_oe,  b'_e = b_e - A_eo A_oo^{-1} b_o,
//   x_o = A_oo^{-1} (b_o - A_oe x_e).
// Written out: Laplacian S = d - H_eo H_oe / d, b'_e = b_e + H_eo b_o / d,
// x_o = (b_o + H_oe x_e) / d; Wilson S = 1 - kappa^2 D_eo D_oe,
// b'_e = b_e + kappa D_eo b_o, x_o = b_o + kappa D_oe x_e.
//
// Half-lattice fields hold the sites of one parity in storage order.  With
// D_0 even, the sites i and i ^ 1 have opposite parities, so site i is entry
// i >> 1 of its parity's half field.  All fields here are in the user layout
// (float64 [nrhs][sites] for the Laplacian, complex128 [nrhs][sites][4][3]
// for Wilson) and all arithmetic is FP64; the hop reproduces the library's
// site operator (same spin projection, links and boundary signs).
#include <algorithm>

#include "pt_common.cuh"

struct EoGeom {
    int D[4];
    int stride[4];
    int N, Nh;
};

static EoGeom make_eo_geom(const int dims[4]) {
    EoGeom g;
    int s = 1;
    for (int mu = 0; mu < 4; ++mu) { g.D[mu] = dims[mu]; g.stride[mu] = s; s *= dims[mu]; }
    g.N = s;
    g.Nh = s / 2;
    return g;
}

// storage index and coordinates of entry h of the half field of parity par
__host__ __device__ __forceinline__ int eo_full_site(const EoGeom &g, int par, int h, int x[4]) {
    const int half0 = g.D[0] >> 1;
    const int q = h / half0;
    const int x0h = h - q * half0;
    x[1] = q % g.D[1];
    const int q2 = q / g.D[1];
    x[2] = q2 % g.D[2];
    x[3] = q2 / g.D[2];
    const int b = (par ^ (x[1] + x[2] + x[3])) & 1;
    x[0] = 2 * x0h + b;
    return 2 * h + b;
}

// storage index of x + s e_mu (s = +1 or -1), periodic
__host__ __device__ __forceinline__ int eo_neighbour(const EoGeom &g, int i, const int x[4], int mu, int s) {
    if (s > 0) return (x[mu] == g.D[mu] - 1) ? i - (g.D[mu] - 1) * g.stride[mu] : i + g.stride[mu];
    return (x[mu] == 0) ? i + (g.D[mu] - 1) * g.stride[mu] : i - g.stride[mu];
}

// a field in the user layout read at a storage index: entry y of a full
// field, or entry y >> 1 of a half field
struct UserField {
    const double *f;
    int half;
    int sites;      // N or N / 2
    __device__ __forceinline__ size_t at(int y) const { return (size_t)(half ? (y >> 1) : y); }
};

// (H psi)(x) for the Wilson hopping term at storage index i, psi read from
// field F of right-hand side r: the library's site operator with the
// neighbour spinors taken from a user-layout full or half field
__device__ __forceinline__ void eo_wilson_hop(const EoGeom &g, const double *U64, int antip, const UserField &F,
                                              int r, int i, const int x[4], Cx<double> acc[4][3]) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) acc[s][a] = Cx<double>{0.0, 0.0};
    const double *base = F.f + (size_t)r * F.sites * 24;
#pragma unroll 1
    for (int mu = 0; mu < 4; ++mu) {
#pragma unroll
        for (int dir = 0; dir < 2; ++dir) {
            const int s = dir == 0 ? 1 : -1;
            const int y = eo_neighbour(g, i, x, mu, s);
            const double sg = dir == 0 ? -1.0 : 1.0;          // (1 - g_mu) forward, (1 + g_mu) backward
            const bool cross = antip && mu == 3 && (dir == 0 ? x[3] == g.D[3] - 1 : x[3] == 0);
            const double eta = cross ? -1.0 : 1.0;
            Cx<double> ps[4][3], h[2][3], uh[2][3], u[3][3];
            const double *p = base + F.at(y) * 24;
#pragma unroll
            for (int c = 0; c < 12; ++c) ps[c / 3][c % 3] = Cx<double>{p[2 * c], p[2 * c + 1]};
            spin_project<double>(mu, sg, ps, h);
            load_link<double, double>(U64, g.N, mu, dir == 0 ? i : y, u);
#pragma unroll
            for (int k = 0; k < 2; ++k)
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    Cx<double> t;
                    if (dir == 0) {                             // U_mu(x) h
                        t = cmul(u[a][0], h[k][0]);
                        t = cadd(t, cmul(u[a][1], h[k][1]));
                        t = cadd(t, cmul(u[a][2], h[k][2]));
                    } else {                                    // U_mu(x - mu)^H h
                        t = cconjmul(u[0][a], h[k][0]);
                        t = cadd(t, cconjmul(u[1][a], h[k][1]));
                        t = cadd(t, cconjmul(u[2][a], h[k][2]));
                    }
                    uh[k][a] = t;
                }
            spin_accumulate<double>(mu, sg, eta, uh, acc);
        }
    }
}

// out[r][h] = alpha self[r][site] + beta (hop src)[r][site] at the sites of
// parity par_out (out is a half field); self may be NULL (alpha ignored)
template <int KIND>
__global__ void __launch_bounds__(128) k_eo_axpby_hop(EoGeom g, const double *U64, int antip, int par_out,
                                                      UserField self, double alpha, UserField src, double beta,
                                                      int nrhs, double *out) {
    const long total = (long)nrhs * g.Nh;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int r = (int)(t / g.Nh), h = (int)(t - (long)r * g.Nh);
        int x[4];
        const int i = eo_full_site(g, par_out, h, x);
        if constexpr (KIND == 0) {
            const double *sb = src.f + (size_t)r * src.sites;
            double hop = 0.0;
#pragma unroll
            for (int mu = 0; mu < 4; ++mu) {
                hop += sb[src.at(eo_neighbour(g, i, x, mu, 1))];
                hop += sb[src.at(eo_neighbour(g, i, x, mu, -1))];
            }
            double v = beta * hop;
            if (self.f) v += alpha * self.f[(size_t)r * self.sites + self.at(i)];
            out[(size_t)r * g.Nh + h] = v;
        } else {
            Cx<double> acc[4][3];
            eo_wilson_hop(g, U64, antip, src, r, i, x, acc);
            double *o = out + ((size_t)r * g.Nh + h) * 24;
            const double *sp = self.f ? self.f + ((size_t)r * self.sites + self.at(i)) * 24 : nullptr;
#pragma unroll
            for (int c = 0; c < 12; ++c) {
                double re = beta * acc[c / 3][c % 3].re, im = beta * acc[c / 3][c % 3].im;
                if (sp) { re += alpha * sp[2 * c]; im += alpha * sp[2 * c + 1]; }
                o[2 * c] = re;
                o[2 * c + 1] = im;
            }
        }
    }
}

// x[r][i] = (even i) x_e[r][i >> 1], (odd i) x_o[r][i >> 1]; reals per site: w
__global__ void k_eo_merge(EoGeom g, int w, const double *xe, const double *xo, int nrhs, double *x) {
    const long total = (long)nrhs * g.N;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int r = (int)(t / g.N), i = (int)(t - (long)r * g.N);
        int c[4];
        int q = i;
        for (int mu = 0; mu < 4; ++mu) { c[mu] = q % g.D[mu]; q /= g.D[mu]; }
        const int par = (c[0] + c[1] + c[2] + c[3]) & 1;
        const double *src = (par ? xo : xe) + ((size_t)r * g.Nh + (i >> 1)) * w;
        double *dst = x + ((size_t)r * g.N + i) * w;
        for (int k = 0; k < w; ++k) dst[k] = src[k];
    }
}

// ---------------------------------------------------------------- host side
static int eo_check(pt_ctx *c, const pt_op *op, int nrhs, const char *fn) {
    PT_CHECK_ARG(c && op && op->ctx == c, "%s: bad context/operator", fn);
    PT_CHECK_ARG(nrhs >= 0 && nrhs <= 65535, "%s: nrhs must be in [0, 65535]", fn);
    for (int mu = 0; mu < 4; ++mu)
        PT_CHECK_ARG(op->dims[mu] % 2 == 0, "%s: every lattice side must be even (side %d is %d)", fn, mu,
                     op->dims[mu]);
    return PT_OK;
}

static int eo_launch(pt_ctx *c, const pt_op *op, const EoGeom &g, int par_out, UserField self, double alpha,
                     UserField src, double beta, int nrhs, double *out) {
    const long total = (long)nrhs * g.Nh;
    const int grid = (int)std::min<long>((total + 127) / 128, 64L * c->num_sms);
    if (op->kind == 0)
        k_eo_axpby_hop<0><<<grid, 128, 0, c->stream>>>(g, nullptr, 0, par_out, self, alpha, src, beta, nrhs, out);
    else
        k_eo_axpby_hop<1><<<grid, 128, 0, c->stream>>>(g, op->U64, op->antip, par_out, self, alpha, src, beta,
                                                       nrhs, out);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}

extern "C" int pt_eo_layout(const int dims[4], int parity, int32_t *site_out, int32_t *nbr_out) {
    PT_CHECK_ARG(dims && site_out && nbr_out, "pt_eo_layout: NULL argument");
    PT_CHECK_ARG(parity == 0 || parity == 1, "pt_eo_layout: parity must be 0 or 1");
    long N = 1;
    for (int mu = 0; mu < 4; ++mu) {
        PT_CHECK_ARG(dims[mu] >= 2 && dims[mu] % 2 == 0, "pt_eo_layout: every side must be even");
        N *= dims[mu];
    }
    PT_CHECK_ARG(N <= (1L << 30), "pt_eo_layout: lattice too large");
    const EoGeom g = make_eo_geom(dims);
    for (int h = 0; h < g.Nh; ++h) {
        int x[4];
        const int i = eo_full_site(g, parity, h, x);
        site_out[h] = i;
        for (int mu = 0; mu < 4; ++mu) {
            nbr_out[(size_t)h * 8 + 2 * mu] = eo_neighbour(g, i, x, mu, 1) >> 1;
            nbr_out[(size_t)h * 8 + 2 * mu + 1] = eo_neighbour(g, i, x, mu, -1) >> 1;
        }
    }
    return PT_OK;
}

extern "C" int pt_eo_schur(pt_ctx *c, const pt_op *op, const double *xe_dev, double *ye_dev, int nrhs) {
    int rc = eo_check(c, op, nrhs, "pt_eo_schur");
    if (rc) return rc;
    if (nrhs == 0) return PT_OK;
    PT_CHECK_ARG(xe_dev && ye_dev && xe_dev != ye_dev, "pt_eo_schur: NULL or aliased fields");
    PT_CUDA(cudaSetDevice(c->device));
    const EoGeom g = make_eo_geom(op->dims);
    const int w = op->kind == 0 ? 1 : 24;
    double *to = nullptr;
    if (cudaMallocAsync((void **)&to, sizeof(double) * (size_t)nrhs * g.Nh * w, c->stream) != cudaSuccess) {
        cudaGetLastError();
        pt_set_error("pt_eo_schur: device allocation failed");
        return PT_ERR_OOM;
    }
    const UserField none{nullptr, 1, g.Nh}, xe{xe_dev, 1, g.Nh}, tof{to, 1, g.Nh};
    const double d = 8.0 + op->m2, k2 = op->kappa * op->kappa;
    rc = eo_launch(c, op, g, 1, none, 0.0, xe, 1.0, nrhs, to);                       // t_o = hop(x_e)
    if (!rc) {
        if (op->kind == 0) rc = eo_launch(c, op, g, 0, xe, d, tof, -1.0 / d, nrhs, ye_dev);
        else rc = eo_launch(c, op, g, 0, xe, 1.0, tof, -k2, nrhs, ye_dev);
    }
    cudaFreeAsync(to, c->stream);
    return rc;
}

extern "C" int pt_eo_prepare(pt_ctx *c, const pt_op *op, const double *b_dev, double *be_dev, int nrhs) {
    int rc = eo_check(c, op, nrhs, "pt_eo_prepare");
    if (rc) return rc;
    if (nrhs == 0) return PT_OK;
    PT_CHECK_ARG(b_dev && be_dev && (const double *)be_dev != b_dev, "pt_eo_prepare: NULL or aliased fields");
    PT_CUDA(cudaSetDevice(c->device));
    const EoGeom g = make_eo_geom(op->dims);
    const UserField b{b_dev, 0, g.N};
    const double beta = op->kind == 0 ? 1.0 / (8.0 + op->m2) : op->kappa;
    return eo_launch(c, op, g, 0, b, 1.0, b, beta, nrhs, be_dev);
}

extern "C" int pt_eo_reconstruct(pt_ctx *c, const pt_op *op, const double *xe_dev, const double *b_dev,
                                 double *x_dev, int nrhs) {
    int rc = eo_check(c, op, nrhs, "pt_eo_reconstruct");
    if (rc) return rc;
    if (nrhs == 0) return PT_OK;
    PT_CHECK_ARG(xe_dev && b_dev && x_dev && x_dev != xe_dev && (const double *)x_dev != b_dev,
                 "pt_eo_reconstruct: NULL or aliased fields");
    PT_CUDA(cudaSetDevice(c->device));
    const EoGeom g = make_eo_geom(op->dims);
    const int w = op->kind == 0 ? 1 : 24;
    double *xo = nullptr;
    if (cudaMallocAsync((void **)&xo, sizeof(double) * (size_t)nrhs * g.Nh * w, c->stream) != cudaSuccess) {
        cudaGetLastError();
        pt_set_error("pt_eo_reconstruct: device allocation failed");
        return PT_ERR_OOM;
    }
    const UserField b{b_dev, 0, g.N}, xe{xe_dev, 1, g.Nh};
    if (op->kind == 0) {
        const double inv_d = 1.0 / (8.0 + op->m2);
        rc = eo_launch(c, op, g, 1, b, inv_d, xe, inv_d, nrhs, xo);
    } else {
        rc = eo_launch(c, op, g, 1, b, 1.0, xe, op->kappa, nrhs, xo);
    }
    if (!rc) {
        const long total = (long)nrhs * g.N;
        const int grid = (int)std::min<long>((total + 255) / 256, 64L * c->num_sms);
        k_eo_merge<<<grid, 256, 0, c->stream>>>(g, w, xe_dev, xo, nrhs, x_dev);
        ++pt_kernel_launch_count;
        const cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) rc = pt_cuda_fail(ce, "k_eo_merge", __FILE__, __LINE__);
    }
    cudaFreeAsync(xo, c->stream);
    return rc;
}
