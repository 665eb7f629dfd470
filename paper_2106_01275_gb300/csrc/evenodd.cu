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
// for Wilson) and all arithmetic is FP64.
//
// The site arithmetic and the sequence of steps are shared by the device
// entry points and host-only ones (which tests run without a GPU): only the
// loop over sites differs (a kernel launch or a host loop).
#include <algorithm>
#include <vector>

#include "eo_geom.cuh"
#include "hd_complex.cuh"
#include "hd_vec.cuh"
#include "hd_wilson.cuh"
#include "pt_common.cuh"

// one output entry: out[r][h] = alpha self[r][site] + beta (hop src)[r][site]
// at the site of parity par_out (out is a half field; self may be NULL)
template <class L>
__host__ __device__ void eo_axpby_site(const EoGeom &g, const L &U, const EoOp &o, int par_out,
                                       const UserField &self, double alpha, const UserField &src, double beta, int r,
                                       int h, double *out) {
    int x[4];
    const int i = eo_full_site(g, par_out, h, x);
    if (o.kind == 0) {
        const double *sb = src.f + (size_t)r * src.sites;
        double hop = 0.0;
        for (int mu = 0; mu < 4; ++mu) {
            hop += sb[src.at(eo_neighbour(g, i, x, mu, 1))];
            hop += sb[src.at(eo_neighbour(g, i, x, mu, -1))];
        }
        double v = beta * hop;
        if (self.f) v += alpha * self.f[(size_t)r * self.sites + self.at(i)];
        out[(size_t)r * g.Nh + h] = v;
    } else {
        zd acc[12];
        eo_wilson_hop(g, U, o, src, r, i, x, acc);
        double *ov = out + ((size_t)r * g.Nh + h) * 24;
        const double *sp = self.f ? self.f + ((size_t)r * self.sites + self.at(i)) * 24 : nullptr;
        for (int c = 0; c < 12; ++c) {
            double re = beta * acc[c].re, im = beta * acc[c].im;
            if (sp) { re += alpha * sp[2 * c]; im += alpha * sp[2 * c + 1]; }
            ov[2 * c] = re;
            ov[2 * c + 1] = im;
        }
    }
}

// x[r][i] = x_e[r][i >> 1] (even i) or x_o[r][i >> 1] (odd i); w reals per site
__host__ __device__ __forceinline__ void eo_merge_site(const EoGeom &g, int w, const double *xe, const double *xo,
                                                       int r, int i, double *x) {
    int q = i, par = 0;
    for (int mu = 0; mu < 4; ++mu) { par += q % g.D[mu]; q /= g.D[mu]; }
    const double *src = ((par & 1) ? xo : xe) + ((size_t)r * g.Nh + (i >> 1)) * w;
    double *dst = x + ((size_t)r * g.N + i) * w;
    for (int k = 0; k < w; ++k) dst[k] = src[k];
}

// ---------------------------------------------------------------- kernels
__global__ void __launch_bounds__(128) k_eo_axpby_hop(EoGeom g, PackedLinks U, EoOp o, int par_out, UserField self,
                                                      double alpha, UserField src, double beta, int nrhs,
                                                      double *out) {
    const long total = (long)nrhs * g.Nh;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int r = (int)(t / g.Nh), h = (int)(t - (long)r * g.Nh);
        eo_axpby_site(g, U, o, par_out, self, alpha, src, beta, r, h, out);
    }
}

__global__ void k_eo_block(EoGeom g, const double *B, int par_out, UserField in, int nrhs, double *out) {
    const long total = (long)nrhs * g.Nh;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int r = (int)(t / g.Nh), h = (int)(t - (long)r * g.Nh);
        eo_block_site(g, B, par_out, in, r, h, out);
    }
}

__global__ void k_eo_merge(EoGeom g, int w, const double *xe, const double *xo, int nrhs, double *x) {
    const long total = (long)nrhs * g.N;
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (long)gridDim.x * blockDim.x) {
        const int r = (int)(t / g.N), i = (int)(t - (long)r * g.N);
        eo_merge_site(g, w, xe, xo, r, i, x);
    }
}

// ---------------------------------------------------------------- executors
// The steps below run the site arithmetic either as kernels on the context
// stream (DevExec) or as host loops (HostExec); both offer the same calls.
struct DevExec : DevVec {
    EoGeom g;
    PackedLinks U;
    EoOp o;
    int hop(int par_out, UserField self, double alpha, UserField src, double beta, int nrhs, double *out) {
        const long total = (long)nrhs * g.Nh;
        const int grid = (int)std::max(1L, std::min((total + 127) / 128, 64L * c->num_sms));
        k_eo_axpby_hop<<<grid, 128, 0, c->stream>>>(g, U, o, par_out, self, alpha, src, beta, nrhs, out);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
    int blk(int par_out, const double *B, UserField in, int nrhs, double *out) {
        const long total = (long)nrhs * g.Nh;
        const int grid = (int)std::max(1L, std::min((total + 127) / 128, 64L * c->num_sms));
        k_eo_block<<<grid, 128, 0, c->stream>>>(g, B, par_out, in, nrhs, out);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
    int merge(int w, const double *xe, const double *xo, int nrhs, double *x) {
        const long total = (long)nrhs * g.N;
        const int grid = (int)std::max(1L, std::min((total + 255) / 256, 64L * c->num_sms));
        k_eo_merge<<<grid, 256, 0, c->stream>>>(g, w, xe, xo, nrhs, x);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
};

struct HostExec : HostVec {
    EoGeom g;
    UserLinks U;
    EoOp o;
    int hop(int par_out, UserField self, double alpha, UserField src, double beta, int nrhs, double *out) {
        for (int r = 0; r < nrhs; ++r)
            for (int h = 0; h < g.Nh; ++h) eo_axpby_site(g, U, o, par_out, self, alpha, src, beta, r, h, out);
        return PT_OK;
    }
    int blk(int par_out, const double *B, UserField in, int nrhs, double *out) {
        for (int r = 0; r < nrhs; ++r)
            for (int h = 0; h < g.Nh; ++h) eo_block_site(g, B, par_out, in, r, h, out);
        return PT_OK;
    }
    int merge(int w, const double *xe, const double *xo, int nrhs, double *x) {
        for (int r = 0; r < nrhs; ++r)
            for (int i = 0; i < g.N; ++i) eo_merge_site(g, w, xe, xo, r, i, x);
        return PT_OK;
    }
};

// ---------------------------------------------------------------- the steps
// Aee, Aoo_inv: the clover Wilson operator's diagonal blocks 1 + C on the even
// sites and the inverses of those on the odd sites ([N/2][12][12] complex, by
// half-field entry), or NULL for the plain operators (A_ee = A_oo = d):
//   S x_e = A_ee x_e - kappa^2 D_eo A_oo^{-1} D_oe x_e,
//   b'_e = b_e + kappa D_eo A_oo^{-1} b_o,  x_o = A_oo^{-1} (b_o + kappa D_oe x_e).
struct EoParams {
    int kind;
    double m2, kappa;
    const double *Aee, *Aoo_inv;
};

template <class X>
static int eo_schur_run(X &ex, const EoParams &P, const double *xe, double *ye, int nrhs) {
    const EoGeom &g = ex.g;
    const int w = P.kind == 0 ? 1 : 24;
    const size_t half = (size_t)nrhs * g.Nh * w;
    double *to = ex.alloc(half * (P.Aoo_inv ? 2 : 1) + (P.Aee ? half : 0));
    if (!to) {
        pt_set_error("pt_eo_schur: allocation of the work fields failed");
        return PT_ERR_OOM;
    }
    const UserField none{nullptr, 1, g.Nh}, xef{xe, 1, g.Nh};
    int rc = ex.hop(1, none, 0.0, xef, 1.0, nrhs, to);                               // t_o = hop(x_e)
    if (!rc && P.kind == 0) {
        const double d = 8.0 + P.m2;
        rc = ex.hop(0, xef, d, UserField{to, 1, g.Nh}, -1.0 / d, nrhs, ye);          // d x_e - hop(t_o) / d
    } else if (!rc) {
        double *uo = to, *we = nullptr;
        if (P.Aoo_inv) {
            uo = to + half;
            rc = ex.blk(1, P.Aoo_inv, UserField{to, 1, g.Nh}, nrhs, uo);             // A_oo^{-1} t_o
        }
        UserField self = xef;
        if (!rc && P.Aee) {
            we = to + half * (P.Aoo_inv ? 2 : 1);
            rc = ex.blk(0, P.Aee, xef, nrhs, we);                                    // A_ee x_e
            self = UserField{we, 1, g.Nh};
        }
        if (!rc) rc = ex.hop(0, self, 1.0, UserField{uo, 1, g.Nh}, -P.kappa * P.kappa, nrhs, ye);
    }
    ex.release(to);
    return rc;
}

template <class X>
static int eo_prepare_run(X &ex, const EoParams &P, const double *b, double *be, int nrhs) {
    const EoGeom &g = ex.g;
    const UserField bf{b, 0, g.N};
    if (P.kind == 0) return ex.hop(0, bf, 1.0, bf, 1.0 / (8.0 + P.m2), nrhs, be);    // b_e + hop(b_o) / d
    if (!P.Aoo_inv) return ex.hop(0, bf, 1.0, bf, P.kappa, nrhs, be);                // b_e + kappa hop(b_o)
    double *uo = ex.alloc((size_t)nrhs * g.Nh * 24);
    if (!uo) {
        pt_set_error("pt_eo_prepare: allocation of the odd half field failed");
        return PT_ERR_OOM;
    }
    int rc = ex.blk(1, P.Aoo_inv, bf, nrhs, uo);                                     // A_oo^{-1} b_o
    if (!rc) rc = ex.hop(0, bf, 1.0, UserField{uo, 1, g.Nh}, P.kappa, nrhs, be);
    ex.release(uo);
    return rc;
}

template <class X>
static int eo_reconstruct_run(X &ex, const EoParams &P, const double *xe, const double *b, double *x, int nrhs) {
    const EoGeom &g = ex.g;
    const int w = P.kind == 0 ? 1 : 24;
    const size_t half = (size_t)nrhs * g.Nh * w;
    double *vo = ex.alloc(half * (P.Aoo_inv ? 2 : 1));
    if (!vo) {
        pt_set_error("pt_eo_reconstruct: allocation of the odd half field failed");
        return PT_ERR_OOM;
    }
    const UserField bf{b, 0, g.N}, xef{xe, 1, g.Nh};
    int rc;
    double *xo = vo;
    if (P.kind == 0) {
        const double inv_d = 1.0 / (8.0 + P.m2);
        rc = ex.hop(1, bf, inv_d, xef, inv_d, nrhs, vo);                             // (b_o + hop(x_e)) / d
    } else {
        rc = ex.hop(1, bf, 1.0, xef, P.kappa, nrhs, vo);                             // b_o + kappa hop(x_e)
        if (!rc && P.Aoo_inv) {
            xo = vo + half;
            rc = ex.blk(1, P.Aoo_inv, UserField{vo, 1, g.Nh}, nrhs, xo);             // A_oo^{-1} (...)
        }
    }
    if (!rc) rc = ex.merge(w, xe, xo, nrhs, x);
    ex.release(vo);
    return rc;
}

// ---------------------------------------------------------------- the even solve
// S x = b' for one right-hand side (even half fields of n reals), from x = 0:
// CG for the Laplacian (S symmetric positive definite), BiCGStab for Wilson
// (restarted from the true residual, as the oracle's).  work: 6 n reals.
// *iters: Krylov iterations; *relres: ||b' - S x|| / ||b'|| recomputed at the
// end.  PT_ERR_NOCONV if the iteration limit is reached first.
template <class X>
static int eo_krylov(X &ex, const EoParams &P, const double *bp, double *x, double *work, double tol, int maxit,
                     int *iters, double *relres) {
    const EoGeom &g = ex.g;
    const int cplx = P.kind == 1;
    const long n = (long)g.Nh * (cplx ? 24 : 1);
    double *r = work, *p = work + n, *q = work + 2 * n, *r0 = work + 3 * n, *s = work + 4 * n, *t = work + 5 * n;
    int rc;
    zd z, z2;
    *iters = 0;
    *relres = 0.0;
    if ((rc = ex.zero(n, x)) || (rc = ex.dot(n, cplx, bp, bp, &z))) return rc;
    const double bn = sqrt(z.re);
    if (bn == 0.0) return PT_OK;
    const double stop = tol * bn;
    bool converged = false;
    if (!cplx) {                                                         // CG
        if ((rc = ex.copy(n, bp, r)) || (rc = ex.copy(n, r, p)) || (rc = ex.dot(n, 0, r, r, &z))) return rc;
        double rr = z.re;
        while (*iters < maxit) {
            if ((rc = eo_schur_run(ex, P, p, q, 1)) || (rc = ex.dot(n, 0, p, q, &z))) return rc;
            if (!(z.re > 0.0)) {
                pt_set_error("even-odd CG: p^T S p = %g is not positive", z.re);
                return PT_ERR_NUMERIC;
            }
            const double alpha = rr / z.re;
            if ((rc = ex.axpy(n, 0, zd{alpha, 0.0}, p, x)) || (rc = ex.axpy(n, 0, zd{-alpha, 0.0}, q, r))) return rc;
            ++*iters;
            if ((rc = ex.dot(n, 0, r, r, &z))) return rc;
            if (sqrt(z.re) <= stop) { converged = true; break; }
            if ((rc = ex.xpay(n, 0, r, zd{z.re / rr, 0.0}, p))) return rc;           // p = r + beta p
            rr = z.re;
        }
    } else {                                                             // BiCGStab
        for (;;) {
            if ((rc = eo_schur_run(ex, P, x, q, 1)) || (rc = ex.copy(n, bp, r)) ||
                (rc = ex.axpy(n, 1, zd{-1.0, 0.0}, q, r)) || (rc = ex.dot(n, 1, r, r, &z)))
                return rc;
            if (sqrt(z.re) <= stop) { converged = true; break; }
            if (*iters >= maxit) break;
            zd rho;
            if ((rc = ex.copy(n, r, r0)) || (rc = ex.copy(n, r, p)) || (rc = ex.dot(n, 1, r0, r, &rho))) return rc;
            while (*iters < maxit) {
                if ((rc = eo_schur_run(ex, P, p, q, 1)) || (rc = ex.dot(n, 1, r0, q, &z))) return rc;   // v = S p
                const zd alpha = zdiv(rho, z);
                if (!isfinite(alpha.re) || !isfinite(alpha.im)) {
                    pt_set_error("even-odd BiCGStab: breakdown (r0^H v = 0)");
                    return PT_ERR_NUMERIC;
                }
                if ((rc = ex.copy(n, r, s)) || (rc = ex.axpy(n, 1, zd{-alpha.re, -alpha.im}, q, s)) ||
                    (rc = eo_schur_run(ex, P, s, t, 1)) || (rc = ex.dot(n, 1, t, t, &z)) ||
                    (rc = ex.dot(n, 1, t, s, &z2)))
                    return rc;
                const zd omega = z.re > 0.0 ? zd{z2.re / z.re, z2.im / z.re} : zd{0.0, 0.0};
                if ((rc = ex.axpy(n, 1, alpha, p, x)) || (rc = ex.axpy(n, 1, omega, s, x)) ||
                    (rc = ex.copy(n, s, r)) || (rc = ex.axpy(n, 1, zd{-omega.re, -omega.im}, t, r)) ||
                    (rc = ex.dot(n, 1, r, r, &z)))
                    return rc;
                ++*iters;
                if (sqrt(z.re) <= stop || (omega.re == 0.0 && omega.im == 0.0)) break;
                zd rho_new;
                if ((rc = ex.dot(n, 1, r0, r, &rho_new))) return rc;
                const zd beta = zmulc(zdiv(rho_new, rho), zdiv(alpha, omega));
                if ((rc = ex.axpy(n, 1, zd{-omega.re, -omega.im}, q, p)) || (rc = ex.xpay(n, 1, r, beta, p)))
                    return rc;                                                          // p = r + beta (p - omega v)
                rho = rho_new;
            }
        }
    }
    // the true residual of the even system
    if ((rc = eo_schur_run(ex, P, x, q, 1)) || (rc = ex.copy(n, bp, r)) ||
        (rc = ex.axpy(n, cplx, zd{-1.0, 0.0}, q, r)) || (rc = ex.dot(n, cplx, r, r, &z)))
        return rc;
    *relres = sqrt(z.re) / bn;
    if (!converged && !(*relres <= tol)) {
        pt_set_error("even-odd solve: %d iterations, relative residual %g", *iters, *relres);
        return PT_ERR_NOCONV;
    }
    return PT_OK;
}

// A x = b for nrhs full fields: b'_e, the even solve per right-hand side, the
// reconstruction.  iters / relres (host, may be NULL): per right-hand side.
template <class X>
static int eo_solve_run(X &ex, const EoParams &P, const double *b, double *x, int nrhs, double tol, int maxit,
                        int *iters, double *relres) {
    const EoGeom &g = ex.g;
    const long n = (long)g.Nh * (P.kind == 1 ? 24 : 1);
    double *be = ex.alloc((size_t)nrhs * n), *xe = ex.alloc((size_t)nrhs * n), *work = ex.alloc((size_t)6 * n);
    double *part = ex.alloc((size_t)2 * VEC_DOT_BLOCKS);
    int rc = PT_OK, rc_nc = PT_OK;
    if (!be || !xe || !work || !part) {
        pt_set_error("even-odd solve: allocation failed");
        rc = PT_ERR_OOM;
    }
    ex.dot_part = part;
    if (!rc) rc = eo_prepare_run(ex, P, b, be, nrhs);
    for (int r = 0; r < nrhs && !rc; ++r) {
        int it = 0;
        double rel = 0.0;
        const int k = eo_krylov(ex, P, be + (size_t)r * n, xe + (size_t)r * n, work, tol, maxit, &it, &rel);
        if (iters) iters[r] = it;
        if (relres) relres[r] = rel;
        if (k == PT_ERR_NOCONV) rc_nc = k;
        else rc = k;
    }
    if (!rc) rc = eo_reconstruct_run(ex, P, xe, b, x, nrhs);
    for (double *q : {part, work, xe, be})
        if (q) ex.release(q);
    return rc ? rc : rc_nc;
}

// ---------------------------------------------------------------- host side
static int eo_check_dims(const int dims[4], const char *fn) {
    PT_CHECK_ARG(dims, "%s: NULL dims", fn);
    long N = 1;
    for (int mu = 0; mu < 4; ++mu) {
        PT_CHECK_ARG(dims[mu] >= 2 && dims[mu] % 2 == 0, "%s: every lattice side must be even (side %d is %d)", fn,
                     mu, dims[mu]);
        N *= dims[mu];
    }
    PT_CHECK_ARG(N <= (1L << 30), "%s: lattice too large", fn);
    return PT_OK;
}

static int eo_dev(pt_ctx *c, const pt_op *op, int nrhs, const char *fn, DevExec *ex, EoParams *P) {
    PT_CHECK_ARG(c && op && op->ctx == c, "%s: bad context/operator", fn);
    PT_CHECK_ARG(nrhs >= 0 && nrhs <= 65535, "%s: nrhs must be in [0, 65535]", fn);
    int rc = eo_check_dims(op->dims, fn);
    if (rc) return rc;
    PT_CUDA(cudaSetDevice(c->device));
    ex->c = c;
    ex->g = make_eo_geom(op->dims);
    ex->U = PackedLinks{op->kind == 1 ? op->U64 : nullptr, ex->g.N};
    ex->o.kind = op->kind;
    ex->o.antip = op->antip;
    ex->o.G = make_gammas();
    P->kind = op->kind;
    P->m2 = op->m2;
    P->kappa = op->kappa;
    P->Aee = P->Aoo_inv = nullptr;
    return PT_OK;
}

static int eo_host(int kind, const int dims[4], double m2, double kappa, const double *U_host, int antip,
                   const char *fn, HostExec *ex, EoParams *P) {
    PT_CHECK_ARG(kind == 0 || kind == 1, "%s: kind must be 0 (Laplacian) or 1 (Wilson)", fn);
    PT_CHECK_ARG(kind == 0 || U_host, "%s: Wilson needs links", fn);
    int rc = eo_check_dims(dims, fn);
    if (rc) return rc;
    ex->g = make_eo_geom(dims);
    ex->U = UserLinks{U_host};
    ex->o.kind = kind;
    ex->o.antip = antip ? 1 : 0;
    ex->o.G = make_gammas();
    P->kind = kind;
    P->m2 = m2;
    P->kappa = kappa;
    P->Aee = P->Aoo_inv = nullptr;
    return PT_OK;
}

extern "C" int pt_eo_layout(const int dims[4], int parity, int32_t *site_out, int32_t *nbr_out) {
    PT_CHECK_ARG(site_out && nbr_out, "pt_eo_layout: NULL argument");
    PT_CHECK_ARG(parity == 0 || parity == 1, "pt_eo_layout: parity must be 0 or 1");
    int rc = eo_check_dims(dims, "pt_eo_layout");
    if (rc) return rc;
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

static int eo_blocks(EoParams *P, const double *Aee, const double *Aoo_inv, const char *fn) {
    PT_CHECK_ARG(P->kind == 1 || (!Aee && !Aoo_inv), "%s: site blocks apply to the Wilson operator only", fn);
    P->Aee = Aee;
    P->Aoo_inv = Aoo_inv;
    return PT_OK;
}

extern "C" int pt_eo_schur(pt_ctx *c, const pt_op *op, const double *Aee_dev, const double *Aoo_inv_dev,
                           const double *xe_dev, double *ye_dev, int nrhs) {
    DevExec ex;
    EoParams P;
    int rc = eo_dev(c, op, nrhs, "pt_eo_schur", &ex, &P);
    if (!rc) rc = eo_blocks(&P, Aee_dev, Aoo_inv_dev, "pt_eo_schur");
    if (rc || nrhs == 0) return rc;
    PT_CHECK_ARG(xe_dev && ye_dev && xe_dev != ye_dev, "pt_eo_schur: NULL or aliased fields");
    return eo_schur_run(ex, P, xe_dev, ye_dev, nrhs);
}

extern "C" int pt_eo_prepare(pt_ctx *c, const pt_op *op, const double *Aoo_inv_dev, const double *b_dev,
                             double *be_dev, int nrhs) {
    DevExec ex;
    EoParams P;
    int rc = eo_dev(c, op, nrhs, "pt_eo_prepare", &ex, &P);
    if (!rc) rc = eo_blocks(&P, nullptr, Aoo_inv_dev, "pt_eo_prepare");
    if (rc || nrhs == 0) return rc;
    PT_CHECK_ARG(b_dev && be_dev && (const double *)be_dev != b_dev, "pt_eo_prepare: NULL or aliased fields");
    return eo_prepare_run(ex, P, b_dev, be_dev, nrhs);
}

extern "C" int pt_eo_reconstruct(pt_ctx *c, const pt_op *op, const double *Aoo_inv_dev, const double *xe_dev,
                                 const double *b_dev, double *x_dev, int nrhs) {
    DevExec ex;
    EoParams P;
    int rc = eo_dev(c, op, nrhs, "pt_eo_reconstruct", &ex, &P);
    if (!rc) rc = eo_blocks(&P, nullptr, Aoo_inv_dev, "pt_eo_reconstruct");
    if (rc || nrhs == 0) return rc;
    PT_CHECK_ARG(xe_dev && b_dev && x_dev && x_dev != xe_dev && (const double *)x_dev != b_dev,
                 "pt_eo_reconstruct: NULL or aliased fields");
    return eo_reconstruct_run(ex, P, xe_dev, b_dev, x_dev, nrhs);
}

// A_ee = 1 + C on the even sites and A_oo^{-1} = (1 + C)^{-1} on the odd ones,
// by half-field entry, from full-lattice blocks C [N][12][12]
__global__ void k_eo_split_blocks(EoGeom g, const double *C, double *Aee, double *Aoo) {
    for (int h = blockIdx.x * blockDim.x + threadIdx.x; h < g.Nh; h += gridDim.x * blockDim.x) {
        for (int par = 0; par < 2; ++par) {
            int x[4];
            const int i = eo_full_site(g, par, h, x);
            const double *src = C + (size_t)i * 288;
            double *dst = (par ? Aoo : Aee) + (size_t)h * 288;
            for (int e = 0; e < 288; ++e) dst[e] = src[e] + ((e & 1) == 0 && (e >> 1) % 13 == 0 && par == 0 ? 1.0 : 0.0);
        }
    }
}

extern "C" int pt_eo_clover_blocks(pt_ctx *c, const pt_op *op, double csw, double *Aee_dev, double *Aoo_inv_dev) {
    PT_CHECK_ARG(c && op && op->ctx == c && op->kind == 1, "pt_eo_clover_blocks: a Wilson operator is required");
    PT_CHECK_ARG(Aee_dev && Aoo_inv_dev && Aee_dev != Aoo_inv_dev, "pt_eo_clover_blocks: NULL or aliased output");
    int rc = eo_check_dims(op->dims, "pt_eo_clover_blocks");
    if (rc) return rc;
    PT_CUDA(cudaSetDevice(c->device));
    const EoGeom g = make_eo_geom(op->dims);
    double *C = nullptr;
    if (cudaMallocAsync((void **)&C, sizeof(double) * 288 * (size_t)g.N, c->stream) != cudaSuccess) {
        cudaGetLastError();
        pt_set_error("pt_eo_clover_blocks: device allocation failed");
        return PT_ERR_OOM;
    }
    rc = pt_clover_blocks(c, op, csw, C);
    double *tmp_o = nullptr;
    if (!rc && cudaMallocAsync((void **)&tmp_o, sizeof(double) * 288 * (size_t)g.Nh, c->stream) != cudaSuccess) {
        cudaGetLastError();
        pt_set_error("pt_eo_clover_blocks: device allocation failed");
        rc = PT_ERR_OOM;
    }
    if (!rc) {
        const int grid = std::max(1, std::min((g.Nh + 127) / 128, 16 * c->num_sms));
        k_eo_split_blocks<<<grid, 128, 0, c->stream>>>(g, C, Aee_dev, tmp_o);
        ++pt_kernel_launch_count;
        const cudaError_t ce = cudaGetLastError();
        if (ce != cudaSuccess) rc = pt_cuda_fail(ce, "k_eo_split_blocks", __FILE__, __LINE__);
    }
    if (!rc) rc = pt_site_blocks_invert(c, g.Nh, tmp_o, 1.0, Aoo_inv_dev);          // (1 + C_oo)^{-1}
    if (tmp_o) cudaFreeAsync(tmp_o, c->stream);
    cudaFreeAsync(C, c->stream);
    return rc;
}

extern "C" int pt_eo_host(int kind, const int dims[4], double m2, double kappa, const double *U_host, int antip,
                          const double *Aee, const double *Aoo_inv, int step, const double *in1, const double *in2,
                          double *out, int nrhs) {
    HostExec ex;
    EoParams P;
    int rc = eo_host(kind, dims, m2, kappa, U_host, antip, "pt_eo_host", &ex, &P);
    if (!rc) rc = eo_blocks(&P, Aee, Aoo_inv, "pt_eo_host");
    if (rc) return rc;
    PT_CHECK_ARG(nrhs >= 0 && in1 && out && (step != 2 || in2), "pt_eo_host: bad argument");
    if (step == 0) return eo_schur_run(ex, P, in1, out, nrhs);
    if (step == 1) return eo_prepare_run(ex, P, in1, out, nrhs);
    PT_CHECK_ARG(step == 2, "pt_eo_host: step must be 0 (Schur), 1 (prepare) or 2 (reconstruct)");
    return eo_reconstruct_run(ex, P, in1, in2, out, nrhs);
}

extern "C" int pt_eo_solve(pt_ctx *c, const pt_op *op, const double *Aee_dev, const double *Aoo_inv_dev,
                           const double *b_dev, double *x_dev, int nrhs, double tol, int maxit, int *iters_out,
                           double *relres_out) {
    DevExec ex;
    EoParams P;
    int rc = eo_dev(c, op, nrhs, "pt_eo_solve", &ex, &P);
    if (!rc) rc = eo_blocks(&P, Aee_dev, Aoo_inv_dev, "pt_eo_solve");
    if (rc || nrhs == 0) return rc;
    PT_CHECK_ARG(b_dev && x_dev && (const double *)x_dev != b_dev, "pt_eo_solve: NULL or aliased fields");
    PT_CHECK_ARG(tol > 0.0 && maxit >= 1, "pt_eo_solve: tol > 0 and maxit >= 1 required");
    rc = eo_solve_run(ex, P, b_dev, x_dev, nrhs, tol, maxit, iters_out, relres_out);
    const cudaError_t ce = cudaStreamSynchronize(c->stream);
    if (!rc && ce != cudaSuccess) rc = pt_cuda_fail(ce, "pt_eo_solve", __FILE__, __LINE__);
    return rc;
}

extern "C" int pt_eo_solve_host(int kind, const int dims[4], double m2, double kappa, const double *U_host,
                                int antip, const double *Aee, const double *Aoo_inv, const double *b, double *x,
                                int nrhs, double tol, int maxit, int *iters_out, double *relres_out) {
    HostExec ex;
    EoParams P;
    int rc = eo_host(kind, dims, m2, kappa, U_host, antip, "pt_eo_solve_host", &ex, &P);
    if (!rc) rc = eo_blocks(&P, Aee, Aoo_inv, "pt_eo_solve_host");
    if (rc) return rc;
    PT_CHECK_ARG(nrhs >= 0 && b && x && tol > 0.0 && maxit >= 1, "pt_eo_solve_host: bad argument");
    return eo_solve_run(ex, P, b, x, nrhs, tol, maxit, iters_out, relres_out);
}
