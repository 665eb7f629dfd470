// Two-level multigrid for the shifted Laplacian as a preconditioner of CG
// (the multigrid part of the solver-fidelity step; the paper solves with an
// adaptive multigrid library, Sec. 4.2, and describes none of its method).
//
// Aggregates are blocks of b^4 sites; the prolongator P holds the normalised
// block indicators, so the Galerkin coarse operator has a closed form:
//   P^T A P = (1 / b) A_coarse(b m^2)
// (per block b^4 (8 + m^2) diagonal terms, 8 b^3 (b - 1) inner hops, b^3 hops
// through each face), i.e. (A_c v)_B = (1 / b) [(8 + b m^2) v_B - sum of the
// eight coarse neighbours].  The two-grid cycle M (nu damped-Jacobi sweeps
// from zero, the coarse correction with A_c solved by CG to 1e-13, nu sweeps)
// is symmetric positive definite, so it preconditions CG.
//
// The per-site arithmetic and the solver are shared by the device entry
// points and host-only twins: only the loop over sites differs.
#include <algorithm>
#include <cmath>
#include <vector>

#include "hd_complex.cuh"
#include "hd_vec.cuh"
#include "pt_common.cuh"

struct MGGeom {
    int D[4], stride[4], N;       // fine lattice
    int C[4], cstride[4], Nc;     // coarse lattice (D / b)
    int b;
    double m2, omega;
};

// storage index of the neighbour of i in direction mu, s = +1 / -1 (periodic)
__host__ __device__ __forceinline__ int mg_step(const int D[4], const int stride[4], int i, int mu, int s) {
    const int x = (i / stride[mu]) % D[mu];
    if (s > 0) return x == D[mu] - 1 ? i - (D[mu] - 1) * stride[mu] : i + stride[mu];
    return x == 0 ? i + (D[mu] - 1) * stride[mu] : i - stride[mu];
}

__host__ __device__ __forceinline__ double mg_nbsum(const int D[4], const int stride[4], const double *v, int i) {
    double s = 0.0;
    for (int mu = 0; mu < 4; ++mu) s += v[mg_step(D, stride, i, mu, 1)] + v[mg_step(D, stride, i, mu, -1)];
    return s;
}

// (A x)_i of the fine operator
__host__ __device__ __forceinline__ double mg_fine_site(const MGGeom &g, const double *x, int i) {
    return (8.0 + g.m2) * x[i] - mg_nbsum(g.D, g.stride, x, i);
}

// (A_c v)_B of the coarse operator (the closed form of P^T A P)
__host__ __device__ __forceinline__ double mg_coarse_site(const MGGeom &g, const double *v, int B) {
    return ((8.0 + g.b * g.m2) * v[B] - mg_nbsum(g.C, g.cstride, v, B)) / g.b;
}

// coarse block of fine site i
__host__ __device__ __forceinline__ int mg_block(const MGGeom &g, int i) {
    int B = 0;
    for (int mu = 3; mu >= 0; --mu) B = B * g.C[mu] + ((i / g.stride[mu]) % g.D[mu]) / g.b;
    return B;
}

// (P^T r)_B = sum over the block's b^4 sites of r, / b^2
__host__ __device__ __forceinline__ double mg_restrict_site(const MGGeom &g, const double *r, int B) {
    int c[4], q = B;
    for (int mu = 0; mu < 4; ++mu) { c[mu] = q % g.C[mu]; q /= g.C[mu]; }
    int base = 0;
    for (int mu = 0; mu < 4; ++mu) base += c[mu] * g.b * g.stride[mu];
    double s = 0.0;
    for (int k3 = 0; k3 < g.b; ++k3)
        for (int k2 = 0; k2 < g.b; ++k2)
            for (int k1 = 0; k1 < g.b; ++k1) {
                const int row = base + k1 * g.stride[1] + k2 * g.stride[2] + k3 * g.stride[3];
                for (int k0 = 0; k0 < g.b; ++k0) s += r[row + k0];
            }
    return s / ((double)g.b * g.b);
}

enum { MG_FINE_APPLY = 0, MG_JACOBI, MG_RESIDUAL, MG_RESTRICT, MG_PROLONG, MG_COARSE_APPLY };

// one site of a step: FINE_APPLY out = A u; JACOBI out = u + omega (w - A u) / (8 + m2);
// RESIDUAL out = w - A u; RESTRICT out (coarse) = P^T u; PROLONG out += P u (u coarse);
// COARSE_APPLY out = A_c u
template <int STEP>
__host__ __device__ __forceinline__ void mg_site(const MGGeom &g, const double *u, const double *w, double *out,
                                                 int i) {
    if constexpr (STEP == MG_FINE_APPLY) out[i] = mg_fine_site(g, u, i);
    else if constexpr (STEP == MG_JACOBI) out[i] = u[i] + g.omega * (w[i] - mg_fine_site(g, u, i)) / (8.0 + g.m2);
    else if constexpr (STEP == MG_RESIDUAL) out[i] = w[i] - mg_fine_site(g, u, i);
    else if constexpr (STEP == MG_RESTRICT) out[i] = mg_restrict_site(g, u, i);
    else if constexpr (STEP == MG_PROLONG) out[i] += u[mg_block(g, i)] / ((double)g.b * g.b);
    else out[i] = mg_coarse_site(g, u, i);
}

template <int STEP>
__global__ void __launch_bounds__(256) k_mg_step(MGGeom g, const double *u, const double *w, double *out, int n) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        mg_site<STEP>(g, u, w, out, i);
}

// ---------------------------------------------------------------- executors
struct MGDev : DevVec {
    MGGeom g;
    template <int STEP>
    int step(const double *u, const double *w, double *out) {
        const int n = (STEP == MG_RESTRICT || STEP == MG_COARSE_APPLY) ? g.Nc : g.N;
        k_mg_step<STEP><<<vgrid(n), 256, 0, c->stream>>>(g, u, w, out, n);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
};

struct MGHost : HostVec {
    MGGeom g;
    template <int STEP>
    int step(const double *u, const double *w, double *out) {
        const int n = (STEP == MG_RESTRICT || STEP == MG_COARSE_APPLY) ? g.Nc : g.N;
        for (int i = 0; i < n; ++i) mg_site<STEP>(g, u, w, out, i);
        return PT_OK;
    }
};

// ---------------------------------------------------------------- the solver
struct MGWork {
    double *ym, *res, *rc, *ec, *cr, *cp, *cq;
};

// A_c e = rc by CG from e = 0 to 1e-13 relative (the coarse solve of M)
template <class X>
static int mg_coarse_solve(X &ex, const MGWork &W) {
    const long n = ex.g.Nc;
    int rc;
    zd z;
    if ((rc = ex.zero(n, W.ec)) || (rc = ex.copy(n, W.rc, W.cr)) || (rc = ex.copy(n, W.cr, W.cp)) ||
        (rc = ex.dot(n, 0, W.cr, W.cr, &z)))
        return rc;
    double rr = z.re;
    const double stop = 1e-26 * rr;
    for (int it = 0; it < 10 * ex.g.Nc + 50 && rr > stop; ++it) {
        if ((rc = ex.template step<MG_COARSE_APPLY>(W.cp, nullptr, W.cq)) || (rc = ex.dot(n, 0, W.cp, W.cq, &z)))
            return rc;
        if (!(z.re > 0.0)) break;
        const double alpha = rr / z.re;
        if ((rc = ex.axpy(n, 0, zd{alpha, 0.0}, W.cp, W.ec)) || (rc = ex.axpy(n, 0, zd{-alpha, 0.0}, W.cq, W.cr)) ||
            (rc = ex.dot(n, 0, W.cr, W.cr, &z)))
            return rc;
        if ((rc = ex.xpay(n, 0, W.cr, zd{z.re / rr, 0.0}, W.cp))) return rc;
        rr = z.re;
    }
    return PT_OK;
}

// out = M r: nu Jacobi sweeps from 0, the coarse correction, nu sweeps
template <class X>
static int mg_cycle(X &ex, int nu, const double *r, double *out, const MGWork &W) {
    const long n = ex.g.N;
    int rc = ex.zero(n, out);
    for (int k = 0; k < nu && !rc; ++k)
        if (!(rc = ex.template step<MG_JACOBI>(out, r, W.ym))) rc = ex.copy(n, W.ym, out);
    if (!rc) rc = ex.template step<MG_RESIDUAL>(out, r, W.res);
    if (!rc) rc = ex.template step<MG_RESTRICT>(W.res, nullptr, W.rc);
    if (!rc) rc = mg_coarse_solve(ex, W);
    if (!rc) rc = ex.template step<MG_PROLONG>(W.ec, nullptr, out);
    for (int k = 0; k < nu && !rc; ++k)
        if (!(rc = ex.template step<MG_JACOBI>(out, r, W.ym))) rc = ex.copy(n, W.ym, out);
    return rc;
}

// A x = b by CG preconditioned with the two-grid cycle, from x = 0, to
// ||b - A x|| <= tol ||b||; work: 4 fine vectors, the cycle's 2 fine and 5
// coarse ones
template <class X>
static int mg_pcg(X &ex, int nu, const double *b, double *x, double tol, int maxit, int *iters, double *relres) {
    const long n = ex.g.N, nc = ex.g.Nc;
    double *r = ex.alloc(n), *z = ex.alloc(n), *p = ex.alloc(n), *q = ex.alloc(n);
    MGWork W{ex.alloc(n), ex.alloc(n), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc)};
    double *part = ex.alloc(2 * VEC_DOT_BLOCKS);
    double *all[] = {r, z, p, q, W.ym, W.res, W.rc, W.ec, W.cr, W.cp, W.cq, part};
    int rc = PT_OK;
    for (double *a : all)
        if (!a) rc = PT_ERR_OOM;
    if (rc) pt_set_error("multigrid solve: allocation failed");
    ex.dot_part = part;
    zd zz;
    *iters = 0;
    *relres = 0.0;
    double bn = 0.0, rz = 0.0;
    bool converged = false;
    if (!rc) rc = ex.zero(n, x);
    if (!rc) rc = ex.dot(n, 0, b, b, &zz);
    if (!rc) bn = sqrt(zz.re);
    if (!rc && bn == 0.0) converged = true;
    if (!rc && !converged) {
        if (!(rc = ex.copy(n, b, r)) && !(rc = mg_cycle(ex, nu, r, z, W)) && !(rc = ex.copy(n, z, p)) &&
            !(rc = ex.dot(n, 0, r, z, &zz)))
            rz = zz.re;
        while (!rc && *iters < maxit) {
            if ((rc = ex.template step<MG_FINE_APPLY>(p, nullptr, q)) || (rc = ex.dot(n, 0, p, q, &zz))) break;
            if (!(zz.re > 0.0)) {
                pt_set_error("multigrid CG: p^T A p = %g is not positive", zz.re);
                rc = PT_ERR_NUMERIC;
                break;
            }
            const double alpha = rz / zz.re;
            if ((rc = ex.axpy(n, 0, zd{alpha, 0.0}, p, x)) || (rc = ex.axpy(n, 0, zd{-alpha, 0.0}, q, r)) ||
                (rc = ex.dot(n, 0, r, r, &zz)))
                break;
            ++*iters;
            if (sqrt(zz.re) <= tol * bn) { converged = true; break; }
            if ((rc = mg_cycle(ex, nu, r, z, W)) || (rc = ex.dot(n, 0, r, z, &zz))) break;
            const double beta = zz.re / rz;
            rz = zz.re;
            if ((rc = ex.xpay(n, 0, z, zd{beta, 0.0}, p))) break;
        }
    }
    if (!rc && bn > 0.0) {                                          // the true residual
        if (!(rc = ex.template step<MG_RESIDUAL>(x, b, r)) && !(rc = ex.dot(n, 0, r, r, &zz)))
            *relres = sqrt(zz.re) / bn;
    }
    for (double *a : all)
        if (a) ex.release(a);
    if (!rc && !converged && !(*relres <= tol)) {
        pt_set_error("multigrid solve: %d iterations, relative residual %g", *iters, *relres);
        rc = PT_ERR_NOCONV;
    }
    return rc;
}

// ---------------------------------------------------------------- entry points
static int mg_geom(const int dims[4], double m2, int block, int nu, double omega, MGGeom *g, const char *fn) {
    PT_CHECK_ARG(dims, "%s: NULL dims", fn);
    PT_CHECK_ARG(block >= 1 && nu >= 0 && nu <= 16 && omega > 0.0 && omega <= 1.0,
                 "%s: block >= 1, 0 <= nu <= 16, 0 < omega <= 1", fn);
    long N = 1;
    int s = 1, cs = 1;
    for (int mu = 0; mu < 4; ++mu) {
        PT_CHECK_ARG(dims[mu] >= 1 && dims[mu] % block == 0, "%s: the block side must divide every lattice side",
                     fn);
        g->D[mu] = dims[mu];
        g->stride[mu] = s;
        g->C[mu] = dims[mu] / block;
        g->cstride[mu] = cs;
        s *= dims[mu];
        cs *= dims[mu] / block;
        N *= dims[mu];
    }
    PT_CHECK_ARG(N <= (1L << 30), "%s: lattice too large", fn);
    g->N = s;
    g->Nc = cs;
    g->b = block;
    g->m2 = m2;
    g->omega = omega;
    return PT_OK;
}

template <class X>
static int mg_solve_all(X &ex, int nu, const double *b, double *x, int nrhs, double tol, int maxit, int *iters_out,
                        double *relres_out) {
    int rc_nc = PT_OK;
    for (int r = 0; r < nrhs; ++r) {
        int it = 0;
        double rel = 0.0;
        const int rc = mg_pcg(ex, nu, b + (size_t)r * ex.g.N, x + (size_t)r * ex.g.N, tol, maxit, &it, &rel);
        if (iters_out) iters_out[r] = it;
        if (relres_out) relres_out[r] = rel;
        if (rc == PT_ERR_NOCONV) rc_nc = rc;
        else if (rc) return rc;
    }
    return rc_nc;
}

extern "C" int pt_mg_solve(pt_ctx *c, const pt_op *op, int block, int nu, double omega, const double *b_dev,
                           double *x_dev, int nrhs, double tol, int maxit, int *iters_out, double *relres_out) {
    PT_CHECK_ARG(c && op && op->ctx == c && op->kind == 0, "pt_mg_solve: a Laplacian operator is required");
    PT_CHECK_ARG(nrhs >= 0 && nrhs <= 65535 && tol > 0.0 && maxit >= 1, "pt_mg_solve: bad nrhs, tol or maxit");
    MGDev ex;
    int rc = mg_geom(op->dims, op->m2, block, nu, omega, &ex.g, "pt_mg_solve");
    if (rc || nrhs == 0) return rc;
    PT_CHECK_ARG(b_dev && x_dev && (const double *)x_dev != b_dev, "pt_mg_solve: NULL or aliased fields");
    PT_CUDA(cudaSetDevice(c->device));
    ex.c = c;
    rc = mg_solve_all(ex, nu, b_dev, x_dev, nrhs, tol, maxit, iters_out, relres_out);
    const cudaError_t ce = cudaStreamSynchronize(c->stream);
    if (!rc && ce != cudaSuccess) rc = pt_cuda_fail(ce, "pt_mg_solve", __FILE__, __LINE__);
    return rc;
}

extern "C" int pt_mg_solve_host(const int dims[4], double m2, int block, int nu, double omega, const double *b,
                                double *x, int nrhs, double tol, int maxit, int *iters_out, double *relres_out) {
    PT_CHECK_ARG(nrhs >= 0 && b && x && tol > 0.0 && maxit >= 1, "pt_mg_solve_host: bad argument");
    MGHost ex;
    int rc = mg_geom(dims, m2, block, nu, omega, &ex.g, "pt_mg_solve_host");
    if (rc) return rc;
    return mg_solve_all(ex, nu, b, x, nrhs, tol, maxit, iters_out, relres_out);
}

extern "C" int pt_mg_cycle_host(const int dims[4], double m2, int block, int nu, double omega, const double *r,
                                double *out) {
    PT_CHECK_ARG(r && out && r != (const double *)out, "pt_mg_cycle_host: NULL or aliased vectors");
    MGHost ex;
    int rc = mg_geom(dims, m2, block, nu, omega, &ex.g, "pt_mg_cycle_host");
    if (rc) return rc;
    const long n = ex.g.N, nc = ex.g.Nc;
    MGWork W{ex.alloc(n), ex.alloc(n), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc)};
    return mg_cycle(ex, nu, r, out, W);
}
