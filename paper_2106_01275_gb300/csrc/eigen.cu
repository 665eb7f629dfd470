// Lowest singular triplets for deflation (Sec. 2.4): block Lanczos with full
// reorthogonalisation on the Hermitian operator H = A (the Laplacian, SPD) or
// H = A^H A = (g5 A)^2 (Wilson-Dirac, g5-Hermitian), then Rayleigh-Ritz.
//
// Vectors live on the device as complex128 [vector][N dof] (the user layout).
// The operator applications are the library's FP64 apply; the block
// operations are two kernels, a Gram matrix X^H Y and a combination
// Y = alpha Y + X C.  Each new vector is orthogonalised twice (classical
// Gram-Schmidt) against the whole basis and dropped when less than 1e-8 of
// its norm is left (the Krylov space holds it already: degenerate spectra);
// the Rayleigh-Ritz eigendecomposition (basis size) runs on the host in FP64.
#include <math.h>

#include <algorithm>
#include <complex>
#include <vector>

#include "pt_common.cuh"

typedef std::complex<double> zc;

// G[i][j] = sum_r conj(X_i[r]) Y_j[r] (G row-major a x b).  One CTA per
// EIG_TI x EIG_TJ tile of G: each thread accumulates the tile over its rows
// (registers), then warp shuffles and a shared-memory pass over the warps,
// in a fixed order.  Each X vector is read ceil(b / EIG_TJ) times, each Y
// vector ceil(a / EIG_TI) times.
#define EIG_TI 4
#define EIG_TJ 8
#define EIG_NT 256
__global__ void __launch_bounds__(EIG_NT) k_eig_gram(long n, const double2 *__restrict__ X, int a,
                                                     const double2 *__restrict__ Y, int b, double2 *G) {
    __shared__ double sh[EIG_NT / 32][2 * EIG_TI * EIG_TJ];
    const int i0 = blockIdx.x * EIG_TI, j0 = blockIdx.y * EIG_TJ;
    const int ni = min(EIG_TI, a - i0), nj = min(EIG_TJ, b - j0);
    double re[EIG_TI][EIG_TJ], im[EIG_TI][EIG_TJ];
#pragma unroll
    for (int ii = 0; ii < EIG_TI; ++ii)
#pragma unroll
        for (int jj = 0; jj < EIG_TJ; ++jj) re[ii][jj] = im[ii][jj] = 0.0;
    for (long r = threadIdx.x; r < n; r += EIG_NT) {
        double2 x[EIG_TI], y[EIG_TJ];
#pragma unroll
        for (int ii = 0; ii < EIG_TI; ++ii) x[ii] = ii < ni ? X[(size_t)(i0 + ii) * n + r] : make_double2(0.0, 0.0);
#pragma unroll
        for (int jj = 0; jj < EIG_TJ; ++jj) y[jj] = jj < nj ? Y[(size_t)(j0 + jj) * n + r] : make_double2(0.0, 0.0);
#pragma unroll
        for (int ii = 0; ii < EIG_TI; ++ii)
#pragma unroll
            for (int jj = 0; jj < EIG_TJ; ++jj) {
                re[ii][jj] += x[ii].x * y[jj].x + x[ii].y * y[jj].y;
                im[ii][jj] += x[ii].x * y[jj].y - x[ii].y * y[jj].x;
            }
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int ii = 0; ii < EIG_TI; ++ii)
#pragma unroll
        for (int jj = 0; jj < EIG_TJ; ++jj) {
            double u = re[ii][jj], v = im[ii][jj];
            for (int o = 16; o > 0; o >>= 1) {
                u += __shfl_down_sync(0xffffffffu, u, o);
                v += __shfl_down_sync(0xffffffffu, v, o);
            }
            if (lane == 0) {
                sh[warp][2 * (ii * EIG_TJ + jj)] = u;
                sh[warp][2 * (ii * EIG_TJ + jj) + 1] = v;
            }
        }
    __syncthreads();
    for (int t = threadIdx.x; t < EIG_TI * EIG_TJ; t += EIG_NT) {
        const int ii = t / EIG_TJ, jj = t % EIG_TJ;
        if (ii >= ni || jj >= nj) continue;
        double u = 0.0, v = 0.0;
        for (int w = 0; w < EIG_NT / 32; ++w) { u += sh[w][2 * t]; v += sh[w][2 * t + 1]; }
        G[(size_t)(i0 + ii) * b + j0 + jj] = make_double2(u, v);
    }
}

// Y_j = alpha Y_j + sum_i X_i C[i][j] (C row-major a x b; Y must not overlap
// X).  A thread owns one row r and EIG_TJ columns (blockIdx.y); C is staged in
// shared memory EIG_CI rows at a time, so each X vector is read
// ceil(b / EIG_TJ) times.  The row loop is uniform over the CTA (barriers).
#define EIG_CI 64
__global__ void __launch_bounds__(EIG_NT) k_eig_combine(long n, const double2 *__restrict__ X, int a,
                                                        const double2 *__restrict__ C, int b, double alpha,
                                                        double2 *Y) {
    __shared__ double2 sc[EIG_CI][EIG_TJ];
    const int j0 = blockIdx.y * EIG_TJ, nj = min(EIG_TJ, b - j0);
    for (long r0 = (long)blockIdx.x * EIG_NT; r0 < n; r0 += (long)gridDim.x * EIG_NT) {
        const long r = r0 + threadIdx.x;
        const bool on = r < n;
        double2 acc[EIG_TJ];
#pragma unroll
        for (int jj = 0; jj < EIG_TJ; ++jj) {
            acc[jj] = make_double2(0.0, 0.0);
            if (on && jj < nj && alpha != 0.0) {
                const double2 yv = Y[(size_t)(j0 + jj) * n + r];
                acc[jj] = make_double2(alpha * yv.x, alpha * yv.y);
            }
        }
        for (int c0 = 0; c0 < a; c0 += EIG_CI) {
            const int nc = min(EIG_CI, a - c0);
            __syncthreads();
            for (int t = threadIdx.x; t < EIG_CI * EIG_TJ; t += EIG_NT) {
                const int ci = t / EIG_TJ, jj = t % EIG_TJ;
                sc[ci][jj] = (ci < nc && jj < nj) ? C[(size_t)(c0 + ci) * b + j0 + jj] : make_double2(0.0, 0.0);
            }
            __syncthreads();
            if (on)
                for (int ci = 0; ci < nc; ++ci) {
                    const double2 x = X[(size_t)(c0 + ci) * n + r];
#pragma unroll
                    for (int jj = 0; jj < EIG_TJ; ++jj) {
                        const double2 c = sc[ci][jj];
                        acc[jj].x += x.x * c.x - x.y * c.y;
                        acc[jj].y += x.x * c.y + x.y * c.x;
                    }
                }
        }
        if (on)
#pragma unroll
            for (int jj = 0; jj < EIG_TJ; ++jj)
                if (jj < nj) Y[(size_t)(j0 + jj) * n + r] = acc[jj];
    }
}

// chiral g5 = diag(1, 1, -1, -1): negate spins 2 and 3 (components 6..11 of a site)
__global__ void k_eig_gamma5(long n_cx, double2 *x) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n_cx; t += (long)gridDim.x * blockDim.x)
        if (t % 12 >= 6) x[t] = make_double2(-x[t].x, -x[t].y);
}

// real parts <-> a real field (the Laplacian's apply takes float64 [nrhs][N])
__global__ void k_eig_re_pack(long n, const double2 *__restrict__ x, double *y) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) y[t] = x[t].x;
}
__global__ void k_eig_re_unpack(long n, const double *__restrict__ y, double2 *x) {
    for (long t = (long)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
        x[t] = make_double2(y[t], 0.0);
}

// ---------------------------------------------------------------- host helpers
// complex products written out (std::complex's operator* may go through a
// NaN-recovering library call on a strict-IEEE host compiler)
static inline zc zmul(zc a, zc b) {
    return zc(a.real() * b.real() - a.imag() * b.imag(), a.real() * b.imag() + a.imag() * b.real());
}
static inline zc zcmul(zc a, zc b) {    // conj(a) b
    return zc(a.real() * b.real() + a.imag() * b.imag(), a.real() * b.imag() - a.imag() * b.real());
}

// Eigenpairs of a Hermitian m x m matrix T (row-major; the Hermitian part
// (T + T^H) / 2 is used): all eigenvalues ascending in w, the eigenvectors of
// the lowest n_vec in X (X[j m + i] = component i of vector j).  Three
// textbook steps (Golub & Van Loan, Matrix Computations, Secs. 8.3.1, 8.3.3):
//  1. Householder reduction to tridiagonal form, A = Q Tc Q^H with
//     Q = H_0 H_1 ... H_{m-3}, H_k = I - 2 v_k v_k^H acting on rows k+1 .. m-1;
//  2. the diagonal unitary D (d_0 = 1, d_{j+1} = d_j beta_j / |beta_j|) makes
//     the sub-diagonal real: Tr = D^H Tc D has sub-diagonal |beta_j|;
//  3. the symmetric QR algorithm with implicit Wilkinson shifts on Tr,
//     Tr = Z diag(w) Z^T, Z the product of the rotations (kept, and applied
//     only for the wanted vectors);
// so eigenvector j of A is Q D z_j.  PT_ERR_NUMERIC if the QR iteration has
// not converged after 60 m steps (NaN input).
static int herm_eig(const std::vector<zc> &T, int m, int n_vec, std::vector<double> &w, std::vector<zc> &X) {
    std::vector<zc> a((size_t)m * m), V((size_t)m * m, zc(0.0, 0.0)), p(m), q(m);
    std::vector<zc> beta(m > 1 ? m - 1 : 1, zc(0.0, 0.0));
    std::vector<char> refl(m, 0);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) a[(size_t)i * m + j] = 0.5 * (T[(size_t)i * m + j] + std::conj(T[(size_t)j * m + i]));
    // 1. Householder: column k below the diagonal -> alpha e_1
    for (int k = 0; k + 2 < m; ++k) {
        const zc x0 = a[(size_t)(k + 1) * m + k];
        double tail = 0.0;
        for (int i = k + 2; i < m; ++i) tail += std::norm(a[(size_t)i * m + k]);
        if (tail == 0.0) { beta[k] = x0; continue; }       // column already reduced
        const double ax0 = std::abs(x0), sigma = sqrt(std::norm(x0) + tail);
        const zc ph = ax0 > 0.0 ? zc(x0.real() / ax0, x0.imag() / ax0) : zc(1.0, 0.0);
        const zc alpha = -sigma * ph;
        zc *v = &V[(size_t)k * m];
        double vn = 0.0;
        for (int i = k + 1; i < m; ++i) v[i] = a[(size_t)i * m + k];
        v[k + 1] -= alpha;
        for (int i = k + 1; i < m; ++i) vn += std::norm(v[i]);
        vn = sqrt(vn);
        for (int i = k + 1; i < m; ++i) v[i] /= vn;
        // trailing block S <- H S H = S - 2 v q^H - 2 q v^H, p = S v, q = p - (v^H p) v;
        // S is kept in its lower triangle (row-major rows: p from rows and their mirror)
        for (int i = k + 1; i < m; ++i) p[i] = zc(0.0, 0.0);
        for (int i = k + 1; i < m; ++i) {
            const zc *row = &a[(size_t)i * m];
            const zc vi = v[i];
            zc acc = zmul(row[i], vi);
            for (int j = k + 1; j < i; ++j) {
                acc += zmul(row[j], v[j]);
                p[j] += zcmul(row[j], vi);             // S_ji = conj(S_ij)
            }
            p[i] += acc;
        }
        double K = 0.0;
        for (int i = k + 1; i < m; ++i) K += zcmul(v[i], p[i]).real();
        for (int i = k + 1; i < m; ++i) q[i] = p[i] - K * v[i];
        for (int i = k + 1; i < m; ++i) {
            zc *row = &a[(size_t)i * m];
            const zc vi = v[i], qi = q[i];
            for (int j = k + 1; j <= i; ++j) row[j] -= 2.0 * (zmul(vi, std::conj(q[j])) + zmul(qi, std::conj(v[j])));
        }
        for (int i = k + 1; i < m; ++i) a[(size_t)i * m + k] = a[(size_t)k * m + i] = zc(0.0, 0.0);
        a[(size_t)(k + 1) * m + k] = alpha;
        a[(size_t)k * m + k + 1] = std::conj(alpha);
        beta[k] = alpha;
        refl[k] = 1;
    }
    if (m >= 2) beta[m - 2] = a[(size_t)(m - 1) * m + m - 2];
    // 2. real tridiagonal Tr: diagonal d, sub-diagonal e; phases D
    std::vector<double> d(m), e(m > 1 ? m - 1 : 1, 0.0);
    std::vector<zc> ph(m, zc(1.0, 0.0));
    for (int i = 0; i < m; ++i) d[i] = a[(size_t)i * m + i].real();
    for (int j = 0; j + 1 < m; ++j) {
        const double r = std::abs(beta[j]);
        e[j] = r;
        ph[j + 1] = r > 0.0 ? zmul(ph[j], zc(beta[j].real() / r, beta[j].imag() / r)) : ph[j];
    }
    // 3. implicit symmetric QR.  Each rotation R_t (plane (k, k+1)) is kept:
    // with Z^T = R_T ... R_1, eigenvector j is row j of Z^T, which the
    // rotations give in reverse order, for the wanted vectors only.
    struct Rot { int k; double c, s; };
    std::vector<Rot> rots;
    rots.reserve((size_t)8 * m);
    const double eps = 2.220446049250313e-16;
    long steps = 0;
    for (;;) {
        for (int i = 0; i + 1 < m; ++i)
            if (fabs(e[i]) <= eps * (fabs(d[i]) + fabs(d[i + 1])) || fabs(e[i]) < 1e-300) e[i] = 0.0;
        int hi = m - 1;
        while (hi > 0 && e[hi - 1] == 0.0) --hi;
        if (hi == 0) break;                     // diagonal
        int lo = hi - 1;
        while (lo > 0 && e[lo - 1] != 0.0) --lo;
        if (++steps > 60L * m) return PT_ERR_NUMERIC;
        // Wilkinson shift: the eigenvalue of the trailing 2 x 2 nearer d[hi]
        const double dd = 0.5 * (d[hi - 1] - d[hi]), bb = e[hi - 1];
        const double mu = d[hi] - bb * bb / (dd + copysign(hypot(dd, bb), dd));
        double x = d[lo] - mu, z = e[lo];
        for (int k = lo; k < hi; ++k) {
            const double r = hypot(x, z);
            const double c = r > 0.0 ? x / r : 1.0, sn = r > 0.0 ? z / r : 0.0;
            if (k > lo) e[k - 1] = r;           // the bulge is chased away
            const double ak = d[k], ak1 = d[k + 1], bk = e[k];
            d[k] = c * c * ak + 2.0 * c * sn * bk + sn * sn * ak1;
            d[k + 1] = sn * sn * ak - 2.0 * c * sn * bk + c * c * ak1;
            e[k] = c * sn * (ak1 - ak) + (c * c - sn * sn) * bk;
            if (k + 1 < hi) {
                z = sn * e[k + 1];              // new bulge at (k + 2, k)
                e[k + 1] *= c;
                x = e[k];
            }
            rots.push_back({k, c, sn});
        }
    }
    std::vector<int> ord(m);
    for (int i = 0; i < m; ++i) ord[i] = i;
    std::sort(ord.begin(), ord.end(), [&](int x, int y) { return d[x] < d[y] || (d[x] == d[y] && x < y); });
    w.resize(m);
    for (int j = 0; j < m; ++j) w[j] = d[ord[j]];
    X.assign((size_t)n_vec * m, zc(0.0, 0.0));
    // z_j^T = e_{ord[j]}^T R_T ... R_1 for all wanted j at once: Zw[i n_vec + j]
    // = component i of z_j, so a rotation updates two contiguous rows
    std::vector<double> Zw((size_t)m * std::max(n_vec, 1), 0.0);
    for (int j = 0; j < n_vec; ++j) Zw[(size_t)ord[j] * n_vec + j] = 1.0;
    for (size_t t = rots.size(); t-- > 0 && n_vec > 0;) {
        const Rot &R = rots[t];
        double *r0 = &Zw[(size_t)R.k * n_vec], *r1 = &Zw[(size_t)(R.k + 1) * n_vec];
        for (int j = 0; j < n_vec; ++j) {
            const double u0 = r0[j], u1 = r1[j];
            r0[j] = R.c * u0 - R.s * u1;
            r1[j] = R.s * u0 + R.c * u1;
        }
    }
    for (int j = 0; j < n_vec; ++j) {
        zc *y = &X[(size_t)j * m];
        for (int i = 0; i < m; ++i) y[i] = Zw[(size_t)i * n_vec + j] * ph[i];
        for (int k = m - 3; k >= 0; --k) {      // y <- H_k y, last reflector first
            if (!refl[k]) continue;
            const zc *v = &V[(size_t)k * m];
            zc s(0.0, 0.0);
            for (int i = k + 1; i < m; ++i) s += zcmul(v[i], y[i]);
            for (int i = k + 1; i < m; ++i) y[i] -= 2.0 * zmul(v[i], s);
        }
    }
    return PT_OK;
}

extern "C" int pt_hermitian_eig(int m, const double *T_host, int n_vec, double *w_out, double *X_out) {
    PT_CHECK_ARG(m >= 1 && m <= 4096, "pt_hermitian_eig: 1 <= m <= 4096");
    PT_CHECK_ARG(n_vec >= 0 && n_vec <= m, "pt_hermitian_eig: 0 <= n_vec <= m");
    PT_CHECK_ARG(T_host && w_out && (n_vec == 0 || X_out), "pt_hermitian_eig: NULL argument");
    std::vector<zc> T((size_t)m * m), X;
    std::vector<double> w;
    for (size_t i = 0; i < (size_t)m * m; ++i) {
        T[i] = zc(T_host[2 * i], T_host[2 * i + 1]);
        if (!std::isfinite(T_host[2 * i]) || !std::isfinite(T_host[2 * i + 1])) {
            pt_set_error("pt_hermitian_eig: non-finite entry");
            return PT_ERR_NUMERIC;
        }
    }
    if (herm_eig(T, m, n_vec, w, X) != PT_OK) {
        pt_set_error("pt_hermitian_eig: the QR iteration did not converge");
        return PT_ERR_NUMERIC;
    }
    for (int j = 0; j < m; ++j) w_out[j] = w[j];
    for (size_t i = 0; i < (size_t)n_vec * m; ++i) {
        X_out[2 * i] = X[i].real();
        X_out[2 * i + 1] = X[i].imag();
    }
    return PT_OK;
}

// ---------------------------------------------------------------- the solver
struct EigRun {
    pt_ctx *c;
    const pt_op *op;
    long n;         // complex entries per vector (N dof)
    int grid;
    double *re_buf; // Laplacian: real fields for the apply
    double2 *tmp;   // Wilson: g5 A x
};

static int eig_gram(const EigRun &E, const double2 *X, int a, const double2 *Y, int b, double2 *d_G,
                    std::vector<zc> &G) {
    const dim3 g((a + EIG_TI - 1) / EIG_TI, (b + EIG_TJ - 1) / EIG_TJ);
    k_eig_gram<<<g, EIG_NT, 0, E.c->stream>>>(E.n, X, a, Y, b, d_G);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    G.resize((size_t)a * b);
    PT_CUDA(cudaMemcpyAsync(G.data(), d_G, (size_t)a * b * sizeof(double2), cudaMemcpyDeviceToHost, E.c->stream));
    PT_CUDA(cudaStreamSynchronize(E.c->stream));
    return PT_OK;
}

static int eig_combine(const EigRun &E, const double2 *X, int a, const std::vector<zc> &C, int b, double alpha,
                       double2 *Y, double2 *d_C) {
    PT_CUDA(cudaMemcpyAsync(d_C, C.data(), (size_t)a * b * sizeof(double2), cudaMemcpyHostToDevice, E.c->stream));
    const dim3 g((unsigned)std::min<long>((E.n + EIG_NT - 1) / EIG_NT, E.grid), (b + EIG_TJ - 1) / EIG_TJ);
    k_eig_combine<<<g, EIG_NT, 0, E.c->stream>>>(E.n, X, a, d_C, b, alpha, Y);
    ++pt_kernel_launch_count;
    PT_CUDA(cudaGetLastError());
    PT_CUDA(cudaStreamSynchronize(E.c->stream));   // C (host) is reused by the caller
    return PT_OK;
}

// Y = H X for b vectors (H = A, or A^H A = g5 A g5 A for Wilson)
static int eig_apply_h(const EigRun &E, const double2 *X, int b, double2 *Y) {
    pt_ctx *c = E.c;
    const long nb = E.n * b;
    if (E.op->kind == 0) {
        k_eig_re_pack<<<E.grid, 256, 0, c->stream>>>(nb, X, E.re_buf);
        int rc = pt_apply(c, E.op, E.re_buf, E.re_buf + nb, b, PT_PREC_FP64);
        if (rc) return rc;
        k_eig_re_unpack<<<E.grid, 256, 0, c->stream>>>(nb, E.re_buf + nb, Y);
        pt_kernel_launch_count += 2;
    } else {
        int rc = pt_apply(c, E.op, (const double *)X, (double *)E.tmp, b, PT_PREC_FP64);
        if (rc) return rc;
        k_eig_gamma5<<<E.grid, 256, 0, c->stream>>>(nb, E.tmp);
        rc = pt_apply(c, E.op, (const double *)E.tmp, (double *)Y, b, PT_PREC_FP64);
        if (rc) return rc;
        k_eig_gamma5<<<E.grid, 256, 0, c->stream>>>(nb, Y);
        pt_kernel_launch_count += 2;
    }
    PT_CUDA(cudaGetLastError());
    return PT_OK;
}

// Append the columns of W (b vectors, overwritten) to the basis B (k
// vectors): the whole block is orthogonalised twice against the basis so far
// (block classical Gram-Schmidt: G = B^H W, W <- W - B G), then each column
// twice against the columns of this block already kept, and normalised,
// unless less than 1e-8 of its norm before the projections remains.  *k grows
// by the columns kept.
static int eig_add_columns(const EigRun &E, double2 *W, int b, double2 *B, int *k, int kmax, double2 *d_G,
                           double2 *d_C) {
    std::vector<zc> G, C(1);
    const int k0 = *k;
    int rc = eig_gram(E, W, b, W, b, d_G, G);
    if (rc) return rc;
    std::vector<double> before(b);
    for (int j = 0; j < b; ++j) before[j] = sqrt(std::max(G[(size_t)j * b + j].real(), 0.0));
    for (int rep = 0; rep < 2 && k0 > 0; ++rep) {
        if ((rc = eig_gram(E, B, k0, W, b, d_G, G))) return rc;
        for (auto &g : G) g = -g;
        if ((rc = eig_combine(E, B, k0, G, b, 1.0, W, d_C))) return rc;
    }
    for (int j = 0; j < b && *k < kmax; ++j) {
        double2 *w = W + (size_t)j * E.n;
        for (int rep = 0; rep < 2 && *k > k0; ++rep) {
            if ((rc = eig_gram(E, B + (size_t)k0 * E.n, *k - k0, w, 1, d_G, G))) return rc;
            for (auto &g : G) g = -g;
            if ((rc = eig_combine(E, B + (size_t)k0 * E.n, *k - k0, G, 1, 1.0, w, d_C))) return rc;
        }
        if ((rc = eig_gram(E, w, 1, w, 1, d_G, G))) return rc;
        const double after = sqrt(std::max(G[0].real(), 0.0));
        if (!(after > 1e-8 * before[j]) || !(after > 0.0)) continue;
        C[0] = 1.0 / after;
        if ((rc = eig_combine(E, w, 1, C, 1, 0.0, B + (size_t)(*k) * E.n, d_C))) return rc;
        ++*k;
    }
    return PT_OK;
}

extern "C" int pt_singular_triplets(pt_ctx *c, const pt_op *op, int n_ev, int block, int n_iter,
                                    const double *start_dev, double *U_dev, double *V_dev, double *s_out) {
    PT_CHECK_ARG(c && op && op->ctx == c, "pt_singular_triplets: bad context/operator");
    PT_CHECK_ARG(start_dev && U_dev && V_dev && s_out, "pt_singular_triplets: NULL argument");
    PT_CHECK_ARG(block >= 1 && block <= 64 && n_iter >= 1 && (long)block * n_iter <= 1024,
                 "pt_singular_triplets: 1 <= block <= 64, basis block * n_iter <= 1024");
    const long n = (long)op->g.N * op->dof;
    PT_CHECK_ARG(n_ev >= 1 && n_ev <= block * n_iter && n_ev <= n, "pt_singular_triplets: bad n_ev");
    PT_CUDA(cudaSetDevice(c->device));
    const int kmax = block * n_iter;
    EigRun E;
    E.c = c;
    E.op = op;
    E.n = n;
    E.grid = 16 * c->num_sms;
    E.re_buf = nullptr;
    E.tmp = nullptr;
    double2 *B = nullptr, *AB = nullptr, *W = nullptr, *d_G = nullptr, *d_C = nullptr;
    const size_t vec_b = (size_t)n * sizeof(double2);
    int rc = PT_OK;
    std::vector<zc> G, C;
    std::vector<double> w;
    std::vector<zc> S;
    int k = 0;                                  // vectors in the basis
    auto fail = [&](int r) { rc = r; };
    do {
        if (cudaMallocAsync((void **)&B, vec_b * kmax, c->stream) != cudaSuccess ||
            cudaMallocAsync((void **)&AB, vec_b * kmax, c->stream) != cudaSuccess ||
            cudaMallocAsync((void **)&W, vec_b * block, c->stream) != cudaSuccess ||
            cudaMallocAsync((void **)&d_G, sizeof(double2) * (size_t)kmax * kmax, c->stream) != cudaSuccess ||
            cudaMallocAsync((void **)&d_C, sizeof(double2) * (size_t)kmax * kmax, c->stream) != cudaSuccess ||
            cudaMallocAsync((void **)&E.re_buf, 2 * sizeof(double) * (size_t)n * block, c->stream) != cudaSuccess ||
            cudaMallocAsync((void **)&E.tmp, vec_b * block, c->stream) != cudaSuccess) {
            cudaGetLastError();
            pt_set_error("pt_singular_triplets: device allocation failed");
            fail(PT_ERR_OOM);
            break;
        }
        // the first candidates: the start block
        if (cudaMemcpyAsync(W, start_dev, vec_b * block, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
            fail(pt_cuda_fail(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__));
            break;
        }
        if (op->kind == 0) {                    // the Laplacian is real: a real start keeps every vector real
            k_eig_re_pack<<<E.grid, 256, 0, c->stream>>>(n * block, W, E.re_buf);
            k_eig_re_unpack<<<E.grid, 256, 0, c->stream>>>(n * block, E.re_buf, W);
            pt_kernel_launch_count += 2;
        }
        int block_in = block;                   // candidate columns in W
        for (int it = 0; it < n_iter; ++it) {
            const int k0 = k;
            if ((rc = eig_add_columns(E, W, block_in, B, &k, kmax, d_G, d_C))) break;
            if (k == k0) break;                 // nothing new: the Krylov space is invariant
            // H applied to the new basis vectors, in chunks of at most `block`
            for (int c0 = k0; c0 < k && !rc; c0 += block)
                rc = eig_apply_h(E, B + (size_t)c0 * n, std::min(block, k - c0), AB + (size_t)c0 * n);
            if (rc) break;
            if (it == n_iter - 1 || k >= kmax || k >= n) break;
            // the next candidates: H times this step's new vectors
            const int nb = std::min(block, k - k0);
            if (cudaMemcpyAsync(W, AB + (size_t)k0 * n, vec_b * nb, cudaMemcpyDeviceToDevice, c->stream) !=
                cudaSuccess) {
                fail(pt_cuda_fail(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__));
                break;
            }
            block_in = nb;
        }
        if (rc) break;
        // Rayleigh-Ritz: T = B^H (H B), eigenpairs ascending, V = B S[:, :n_ev]
        if ((rc = eig_gram(E, B, k, AB, k, d_G, G))) break;
        if (k < n_ev) { pt_set_error("pt_singular_triplets: basis smaller than n_ev"); fail(PT_ERR_NUMERIC); break; }
        const int ne = n_ev;
        if (herm_eig(G, k, ne, w, S) != PT_OK) {
            pt_set_error("pt_singular_triplets: Rayleigh-Ritz eigensolver did not converge");
            fail(PT_ERR_NUMERIC);
            break;
        }
        C.assign((size_t)k * ne, zc(0.0, 0.0));
        for (int j = 0; j < ne; ++j)
            for (int i = 0; i < k; ++i) C[(size_t)i * ne + j] = S[(size_t)j * k + i];
        if ((rc = eig_combine(E, B, k, C, ne, 0.0, (double2 *)V_dev, d_C))) break;
        // singular values and left vectors: Laplacian (SPD) U = V, s = eigenvalue;
        // Wilson s = sqrt(eigenvalue of A^H A) = |A v|, U = A V / s
        if (op->kind == 0) {
            for (int j = 0; j < ne; ++j) s_out[j] = w[j];
            if (cudaMemcpyAsync(U_dev, V_dev, vec_b * ne, cudaMemcpyDeviceToDevice, c->stream) != cudaSuccess) {
                fail(pt_cuda_fail(cudaGetLastError(), "cudaMemcpyAsync", __FILE__, __LINE__));
                break;
            }
        } else {
            for (int j0 = 0; j0 < ne && !rc; j0 += block) {
                const int nb = std::min(block, ne - j0);
                rc = pt_apply(c, op, V_dev + (size_t)j0 * n * 2, (double *)W, nb, PT_PREC_FP64);
                if (rc) break;
                if ((rc = eig_gram(E, W, nb, W, nb, d_G, G))) break;
                std::vector<zc> D((size_t)nb * nb, zc(0.0, 0.0));
                for (int j = 0; j < nb; ++j) {
                    const double sj = sqrt(std::max(G[(size_t)j * nb + j].real(), 0.0));
                    s_out[j0 + j] = sj;
                    D[(size_t)j * nb + j] = sj > 0.0 ? 1.0 / sj : 0.0;
                }
                rc = eig_combine(E, W, nb, D, nb, 0.0, (double2 *)U_dev + (size_t)j0 * n, d_C);
            }
        }
    } while (0);
    if (B) cudaFreeAsync(B, c->stream);
    if (AB) cudaFreeAsync(AB, c->stream);
    if (W) cudaFreeAsync(W, c->stream);
    if (d_G) cudaFreeAsync(d_G, c->stream);
    if (d_C) cudaFreeAsync(d_C, c->stream);
    if (E.re_buf) cudaFreeAsync(E.re_buf, c->stream);
    if (E.tmp) cudaFreeAsync(E.tmp, c->stream);
    cudaStreamSynchronize(c->stream);
    return rc;
}
