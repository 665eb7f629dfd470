// Two-level adaptive aggregation multigrid for the Wilson-Dirac operator as a
// right preconditioner of FGMRES (the solver-fidelity step: the paper solves
// with an adaptive multigrid library, Sec. 4.2, and describes none of its
// method; this is the textbook construction).
//
//   aggregates   blocks of b^4 sites, each split by chirality (spins 0-1 and
//                2-3), so that the prolongator commutes with g5;
//   near-null    nv vectors: counter-based random vectors relaxed by damped
//                Richardson sweeps on A v = 0;
//   prolongator  per aggregate, the near-null vectors restricted to it and
//                orthonormalised (modified Gram-Schmidt); P [N 12, Nc 2 nv];
//   coarse op    A_c = P^H A P as a nine-point block stencil on the coarse
//                lattice (self and the eight neighbours, blocks 2 nv x 2 nv),
//                assembled from the fine hops that stay in or leave a block;
//   cycle        nu damped-Richardson sweeps from zero, the coarse correction
//                (A_c solved by BiCGStab to 1e-10), nu sweeps;
//   outer        FGMRES(m) (the coarse solve is inexact, so the cycle is not a
//                fixed linear map).
//
// With c_sw != 0 the operator is the clover one, A = A_W + C (the site blocks
// of clover.cu in the fine apply, P^H C P in the coarse self blocks).
// All arithmetic FP64, fields in the user layout (complex128 [N][4][3]).  The
// per-site arithmetic and the solver are shared by the device entry point and
// a host-only twin: only the loop over sites differs.
#include <algorithm>
#include <cmath>
#include <vector>

#include "eo_geom.cuh"
#include "hd_complex.cuh"
#include "hd_vec.cuh"
#include "hd_wilson.cuh"
#include "pt_common.cuh"

#define WMG_MAXNV 8

struct WMG {
    EoGeom g;                    // fine lattice
    int C[4], cstride[4], Nc;    // coarse lattice
    int b, bs, nv;               // block side, sites per block, vectors per aggregate
    double kappa, omega;
    EoOp o;                      // gammas and the time boundary
    const double *Cb;            // clover site blocks [N][12][12] complex, or NULL (plain Wilson)
    __host__ __device__ int dc() const { return 2 * nv; }   // coarse degrees of freedom per coarse site
};

// coarse site of fine site i and the site's index inside its block
__host__ __device__ __forceinline__ void wmg_block(const WMG &m, int i, int *B, int *sl) {
    int Bi = 0, s = 0;
    for (int mu = 3; mu >= 0; --mu) {
        const int x = (i / m.g.stride[mu]) % m.g.D[mu];
        Bi = Bi * m.C[mu] + x / m.b;
        s = s * m.b + x % m.b;
    }
    *B = Bi;
    *sl = s;
}

// fine site of (coarse site B, index sl inside the block)
__host__ __device__ __forceinline__ int wmg_site(const WMG &m, int B, int sl) {
    int i = 0, q = B, r = sl;
    for (int mu = 0; mu < 4; ++mu) {
        const int c = q % m.C[mu], k = r % m.b;
        q /= m.C[mu];
        r /= m.b;
        i += (c * m.b + k) * m.g.stride[mu];
    }
    return i;
}

// coarse neighbour in stencil slot d (0 self; 1 + 2 mu + 0 / 1: +mu / -mu)
__host__ __device__ __forceinline__ int wmg_cnb(const WMG &m, int B, int d) {
    if (d == 0) return B;
    const int mu = (d - 1) >> 1, s = ((d - 1) & 1) ? -1 : 1;
    const int x = (B / m.cstride[mu]) % m.C[mu];
    if (s > 0) return x == m.C[mu] - 1 ? B - (m.C[mu] - 1) * m.cstride[mu] : B + m.cstride[mu];
    return x == 0 ? B + (m.C[mu] - 1) * m.cstride[mu] : B - m.cstride[mu];
}

// entry of the prolongator: column (B, a, k), row (site sl of B, component c of half a)
__host__ __device__ __forceinline__ size_t wmg_pidx(const WMG &m, int B, int a, int k, int sl, int c6) {
    return ((((size_t)B * 2 + a) * m.nv + k) * m.bs + sl) * 6 + c6;
}

// (A x)_i = x_i - kappa (H x)_i, 12 complex components
__host__ __device__ __forceinline__ void wmg_apply_site(const WMG &m, const UserLinks &U0, const PackedLinks &U1,
                                                        int packed, const double *x, int i, zd out[12]) {
    int xc[4];
    int q = i;
    for (int mu = 0; mu < 4; ++mu) { xc[mu] = q % m.g.D[mu]; q /= m.g.D[mu]; }
    const UserField F{x, 0, m.g.N};
    zd acc[12];
    if (packed) eo_wilson_hop(m.g, U1, m.o, F, 0, i, xc, acc);
    else eo_wilson_hop(m.g, U0, m.o, F, 0, i, xc, acc);
    const double *xi = x + (size_t)i * 24;
    for (int c = 0; c < 12; ++c) out[c] = zsub(zd{xi[2 * c], xi[2 * c + 1]}, zscal(acc[c], m.kappa));
    if (m.Cb) {                                          // + C(x) x(x)
        const double *Ci = m.Cb + (size_t)i * 288;
        for (int r = 0; r < 12; ++r)
            for (int c = 0; c < 12; ++c)
                out[r] = zadd(out[r], zmulc(zd{Ci[(r * 12 + c) * 2], Ci[(r * 12 + c) * 2 + 1]}, zd{xi[2 * c], xi[2 * c + 1]}));
    }
}

// counter-based start vector k: components uniform in [-1, 1) (SplitMix64 outputs)
__host__ __device__ __forceinline__ double wmg_uniform(uint64_t key, uint64_t c) {
    return (double)(pt_mix64(key + (c + 1ULL) * PT_GAMMA) >> 11) * (2.0 / 9007199254740992.0) - 1.0;
}

enum { WMG_APPLY = 0, WMG_RICHARDSON, WMG_RESIDUAL, WMG_PROLONG, WMG_FILL, WMG_RANDOM };

// one fine site of a step (u, w inputs, out output, all [N][12] complex):
//   APPLY out = A u;  RICHARDSON out = u + omega (w - A u);  RESIDUAL out = w - A u;
//   PROLONG out += P u (u coarse);  FILL P[., ., k] = restriction of u (vector k);
//   RANDOM out = start vector k
template <int STEP>
__host__ __device__ __forceinline__ void wmg_fine(const WMG &m, const UserLinks &U0, const PackedLinks &U1, int packed,
                                                  const double *u, const double *w, double *out, double *P, int k,
                                                  uint64_t key, int i) {
    double *o = out ? out + (size_t)i * 24 : nullptr;
    if constexpr (STEP == WMG_APPLY || STEP == WMG_RICHARDSON || STEP == WMG_RESIDUAL) {
        zd ax[12];
        wmg_apply_site(m, U0, U1, packed, u, i, ax);
        for (int c = 0; c < 12; ++c) {
            zd v = ax[c];
            if constexpr (STEP == WMG_RICHARDSON) {
                const zd wv = w ? zd{w[(size_t)i * 24 + 2 * c], w[(size_t)i * 24 + 2 * c + 1]} : zd{0.0, 0.0};
                v = zadd(zd{u[(size_t)i * 24 + 2 * c], u[(size_t)i * 24 + 2 * c + 1]}, zscal(zsub(wv, ax[c]), m.omega));
            } else if constexpr (STEP == WMG_RESIDUAL) {
                v = zsub(zd{w[(size_t)i * 24 + 2 * c], w[(size_t)i * 24 + 2 * c + 1]}, ax[c]);
            }
            o[2 * c] = v.re;
            o[2 * c + 1] = v.im;
        }
    } else if constexpr (STEP == WMG_PROLONG) {
        int B, sl;
        wmg_block(m, i, &B, &sl);
        const double *uc = u + (size_t)B * m.dc() * 2;
        for (int c = 0; c < 12; ++c) {
            const int a = c / 6, c6 = c % 6;
            zd s = {0.0, 0.0};
            for (int kk = 0; kk < m.nv; ++kk) {
                const size_t pi = wmg_pidx(m, B, a, kk, sl, c6) * 2;
                const int col = a * m.nv + kk;
                s = zadd(s, zmulc(zd{P[pi], P[pi + 1]}, zd{uc[2 * col], uc[2 * col + 1]}));
            }
            o[2 * c] += s.re;
            o[2 * c + 1] += s.im;
        }
    } else if constexpr (STEP == WMG_FILL) {
        int B, sl;
        wmg_block(m, i, &B, &sl);
        for (int c = 0; c < 12; ++c) {
            const size_t pi = wmg_pidx(m, B, c / 6, k, sl, c % 6) * 2;
            P[pi] = u[(size_t)i * 24 + 2 * c];
            P[pi + 1] = u[(size_t)i * 24 + 2 * c + 1];
        }
    } else {
        for (int c = 0; c < 24; ++c) o[c] = wmg_uniform(key, (uint64_t)i * 24 + c);
    }
}

// rc[t] = (P^H r)_t for coarse dof t = (B, a, k): sum over the aggregate of conj(P) r
__host__ __device__ __forceinline__ void wmg_restrict(const WMG &m, const double *P, const double *r, double *rc,
                                                      int t) {
    const int B = t / m.dc(), col = t % m.dc(), a = col / m.nv, k = col % m.nv;
    zd s = {0.0, 0.0};
    for (int sl = 0; sl < m.bs; ++sl) {
        const double *ri = r + (size_t)wmg_site(m, B, sl) * 24 + a * 12;
        for (int c6 = 0; c6 < 6; ++c6) {
            const size_t pi = wmg_pidx(m, B, a, k, sl, c6) * 2;
            s = zadd(s, zmulc(zd{P[pi], -P[pi + 1]}, zd{ri[2 * c6], ri[2 * c6 + 1]}));
        }
    }
    rc[2 * t] = s.re;
    rc[2 * t + 1] = s.im;
}

// orthonormalise the nv columns of aggregate (B, a) by modified Gram-Schmidt,
// twice; returns false if a column vanishes
__host__ __device__ __forceinline__ bool wmg_ortho(const WMG &m, double *P, int B, int a) {
    const int len = m.bs * 6;
    for (int pass = 0; pass < 2; ++pass)
        for (int k = 0; k < m.nv; ++k) {
            double *pk = P + wmg_pidx(m, B, a, k, 0, 0) * 2;
            for (int j = 0; j < k; ++j) {
                const double *pj = P + wmg_pidx(m, B, a, j, 0, 0) * 2;
                zd h = {0.0, 0.0};
                for (int e = 0; e < len; ++e) h = zadd(h, zmulc(zd{pj[2 * e], -pj[2 * e + 1]}, zd{pk[2 * e], pk[2 * e + 1]}));
                for (int e = 0; e < len; ++e) {
                    const zd v = zsub(zd{pk[2 * e], pk[2 * e + 1]}, zmulc(h, zd{pj[2 * e], pj[2 * e + 1]}));
                    pk[2 * e] = v.re;
                    pk[2 * e + 1] = v.im;
                }
            }
            double nrm = 0.0;
            for (int e = 0; e < 2 * len; ++e) nrm += pk[e] * pk[e];
            nrm = sqrt(nrm);
            if (!(nrm > 0.0)) return false;
            for (int e = 0; e < 2 * len; ++e) pk[e] /= nrm;
        }
    return true;
}

// -kappa times one hop of H at site i (coordinates xc) applied to the spinor
// psi of its neighbour in direction mu (dir 0 forward: (1 - g_mu) U_mu(x) psi;
// dir 1 backward: (1 + g_mu) U_mu(x - mu)^H psi), boundary sign included
template <class L>
__host__ __device__ __forceinline__ void wmg_hop_term(const WMG &m, const L &U, int i, const int xc[4], int mu,
                                                      int dir, const zd psi[12], zd out[12]) {
    const int y = eo_neighbour(m.g, i, xc, mu, dir == 0 ? 1 : -1);
    const bool cross = m.o.antip && mu == 3 && (dir == 0 ? xc[3] == m.g.D[3] - 1 : xc[3] == 0);
    const double eta = cross ? -1.0 : 1.0, sgn = dir == 0 ? -1.0 : 1.0;
    zd chi[12];
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            zd t = {0.0, 0.0};
            for (int b = 0; b < 3; ++b) {
                const zd w = dir == 0 ? U(i, mu, a * 3 + b) : zconj(U(y, mu, b * 3 + a));
                t = zadd(t, zmulc(w, psi[s * 3 + b]));
            }
            chi[s * 3 + a] = t;
        }
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            zd gchi = {0.0, 0.0};
            for (int t = 0; t < 4; ++t) gchi = zadd(gchi, zmulc(m.o.G.g[mu][s * 4 + t], chi[t * 3 + a]));
            out[s * 3 + a] = zscal(zadd(chi[s * 3 + a], zscal(gchi, sgn)), -m.kappa * eta);
        }
}

// the nine stencil blocks of A_c = P^H A P at coarse site B:
// Ac[((B 9 + d) dc + row) dc + col], d as in wmg_cnb
template <class L>
__host__ __device__ void wmg_build_site(const WMG &m, const L &U, const double *P, double *Ac, int B) {
    const int dc = m.dc();
    double *A = Ac + (size_t)B * 9 * dc * dc * 2;
    for (int e = 0; e < 9 * dc * dc * 2; ++e) A[e] = 0.0;
    for (int sl = 0; sl < m.bs; ++sl) {
        const int i = wmg_site(m, B, sl);
        int xc[4], q = i;
        for (int mu = 0; mu < 4; ++mu) { xc[mu] = q % m.g.D[mu]; q /= m.g.D[mu]; }
        // the identity part of A: P_row^H P_col over this site
        for (int a = 0; a < 2; ++a)
            for (int kr = 0; kr < m.nv; ++kr)
                for (int kc = 0; kc < m.nv; ++kc) {
                    zd s = {0.0, 0.0};
                    for (int c6 = 0; c6 < 6; ++c6) {
                        const size_t pr = wmg_pidx(m, B, a, kr, sl, c6) * 2, pc = wmg_pidx(m, B, a, kc, sl, c6) * 2;
                        s = zadd(s, zmulc(zd{P[pr], -P[pr + 1]}, zd{P[pc], P[pc + 1]}));
                    }
                    double *e = A + ((size_t)(a * m.nv + kr) * dc + a * m.nv + kc) * 2;
                    e[0] += s.re;
                    e[1] += s.im;
                }
        // the clover term (site-local): P_row^H C(x) P_col, into the self slot
        if (m.Cb) {
            const double *Ci = m.Cb + (size_t)i * 288;
            for (int ar = 0; ar < 2; ++ar)
                for (int kr = 0; kr < m.nv; ++kr)
                    for (int ac = 0; ac < 2; ++ac)
                        for (int kc = 0; kc < m.nv; ++kc) {
                            zd s = {0.0, 0.0};
                            for (int cr = 0; cr < 6; ++cr) {
                                zd t = {0.0, 0.0};
                                for (int cc = 0; cc < 6; ++cc) {
                                    const size_t pc = wmg_pidx(m, B, ac, kc, sl, cc) * 2;
                                    const size_t ci = ((size_t)(ar * 6 + cr) * 12 + ac * 6 + cc) * 2;
                                    t = zadd(t, zmulc(zd{Ci[ci], Ci[ci + 1]}, zd{P[pc], P[pc + 1]}));
                                }
                                const size_t pr = wmg_pidx(m, B, ar, kr, sl, cr) * 2;
                                s = zadd(s, zmulc(zd{P[pr], -P[pr + 1]}, t));
                            }
                            double *e = A + ((size_t)(ar * m.nv + kr) * dc + ac * m.nv + kc) * 2;
                            e[0] += s.re;
                            e[1] += s.im;
                        }
        }
        // the hops: inside the block -> slot 0, across a face -> the direction's slot
        for (int mu = 0; mu < 4; ++mu)
            for (int dir = 0; dir < 2; ++dir) {
                const int y = eo_neighbour(m.g, i, xc, mu, dir == 0 ? 1 : -1);
                const int lx = xc[mu] % m.b;
                const bool inside = dir == 0 ? lx != m.b - 1 : lx != 0;
                const int slot = inside ? 0 : 1 + 2 * mu + dir;
                int By, sly;
                wmg_block(m, y, &By, &sly);
                for (int ac = 0; ac < 2; ++ac)
                    for (int kc = 0; kc < m.nv; ++kc) {
                        zd psi[12], h[12];
                        for (int c = 0; c < 12; ++c) psi[c] = {0.0, 0.0};
                        for (int c6 = 0; c6 < 6; ++c6) {
                            const size_t pc = wmg_pidx(m, By, ac, kc, sly, c6) * 2;
                            psi[ac * 6 + c6] = zd{P[pc], P[pc + 1]};
                        }
                        wmg_hop_term(m, U, i, xc, mu, dir, psi, h);
                        for (int ar = 0; ar < 2; ++ar)
                            for (int kr = 0; kr < m.nv; ++kr) {
                                zd s = {0.0, 0.0};
                                for (int c6 = 0; c6 < 6; ++c6) {
                                    const size_t pr = wmg_pidx(m, B, ar, kr, sl, c6) * 2;
                                    s = zadd(s, zmulc(zd{P[pr], -P[pr + 1]}, h[ar * 6 + c6]));
                                }
                                double *e = A + (((size_t)slot * dc + ar * m.nv + kr) * dc + ac * m.nv + kc) * 2;
                                e[0] += s.re;
                                e[1] += s.im;
                            }
                    }
            }
    }
}

// (A_c v)_B = sum over the nine slots of Ac[B][d] v[neighbour(B, d)]
__host__ __device__ __forceinline__ void wmg_capply(const WMG &m, const double *Ac, const double *v, double *out,
                                                    int B) {
    const int dc = m.dc();
    const double *A = Ac + (size_t)B * 9 * dc * dc * 2;
    for (int row = 0; row < dc; ++row) {
        zd s = {0.0, 0.0};
        for (int d = 0; d < 9; ++d) {
            const double *vn = v + (size_t)wmg_cnb(m, B, d) * dc * 2;
            const double *ar = A + ((size_t)d * dc + row) * dc * 2;
            for (int col = 0; col < dc; ++col)
                s = zadd(s, zmulc(zd{ar[2 * col], ar[2 * col + 1]}, zd{vn[2 * col], vn[2 * col + 1]}));
        }
        out[(size_t)B * dc * 2 + 2 * row] = s.re;
        out[(size_t)B * dc * 2 + 2 * row + 1] = s.im;
    }
}

// ---------------------------------------------------------------- kernels
template <int STEP>
__global__ void __launch_bounds__(128) k_wmg_fine(WMG m, PackedLinks U1, const double *u, const double *w,
                                                  double *out, double *P, int k, uint64_t key) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m.g.N; i += gridDim.x * blockDim.x)
        wmg_fine<STEP>(m, UserLinks{nullptr}, U1, 1, u, w, out, P, k, key, i);
}
__global__ void k_wmg_restrict(WMG m, const double *P, const double *r, double *rc) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.Nc * m.dc(); t += gridDim.x * blockDim.x)
        wmg_restrict(m, P, r, rc, t);
}
__global__ void k_wmg_ortho(WMG m, double *P, int *bad) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < m.Nc * 2; t += gridDim.x * blockDim.x)
        if (!wmg_ortho(m, P, t / 2, t % 2)) atomicAdd(bad, 1);
}
__global__ void k_wmg_build(WMG m, PackedLinks U1, const double *P, double *Ac) {
    for (int B = blockIdx.x * blockDim.x + threadIdx.x; B < m.Nc; B += gridDim.x * blockDim.x)
        wmg_build_site(m, U1, P, Ac, B);
}
__global__ void k_wmg_capply(WMG m, const double *Ac, const double *v, double *out) {
    for (int B = blockIdx.x * blockDim.x + threadIdx.x; B < m.Nc; B += gridDim.x * blockDim.x)
        wmg_capply(m, Ac, v, out, B);
}

// ---------------------------------------------------------------- executors
struct WMGDev : DevVec {
    WMG m;
    PackedLinks U1;
    double *P = nullptr, *Ac = nullptr;
    int grid(long n, int nt) const { return (int)std::max(1L, std::min((n + nt - 1) / nt, 16L * c->num_sms)); }
    template <int STEP>
    int fine(const double *u, const double *w, double *out, int k = 0, uint64_t key = 0) {
        k_wmg_fine<STEP><<<grid(m.g.N, 128), 128, 0, c->stream>>>(m, U1, u, w, out, P, k, key);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
    int restrict_(const double *r, double *rc) {
        k_wmg_restrict<<<grid((long)m.Nc * m.dc(), 128), 128, 0, c->stream>>>(m, P, r, rc);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
    int ortho() {
        int *bad = nullptr, h_bad = 0;
        if (cudaMallocAsync((void **)&bad, sizeof(int), c->stream) != cudaSuccess) {
            cudaGetLastError();
            return PT_ERR_OOM;
        }
        cudaError_t ce = cudaMemsetAsync(bad, 0, sizeof(int), c->stream);
        if (ce == cudaSuccess) {
            k_wmg_ortho<<<grid((long)m.Nc * 2, 64), 64, 0, c->stream>>>(m, P, bad);
            ++pt_kernel_launch_count;
            ce = cudaGetLastError();
        }
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&h_bad, bad, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(c->stream);
        cudaFreeAsync(bad, c->stream);
        if (ce != cudaSuccess) return pt_cuda_fail(ce, "k_wmg_ortho", __FILE__, __LINE__);
        return h_bad ? PT_ERR_NUMERIC : PT_OK;
    }
    int build() {
        k_wmg_build<<<grid(m.Nc, 64), 64, 0, c->stream>>>(m, U1, P, Ac);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
    int capply(const double *v, double *out) {
        k_wmg_capply<<<grid(m.Nc, 64), 64, 0, c->stream>>>(m, Ac, v, out);
        ++pt_kernel_launch_count;
        PT_CUDA(cudaGetLastError());
        return PT_OK;
    }
};

struct WMGHost : HostVec {
    WMG m;
    UserLinks U0;
    double *P = nullptr, *Ac = nullptr;
    template <int STEP>
    int fine(const double *u, const double *w, double *out, int k = 0, uint64_t key = 0) {
        for (int i = 0; i < m.g.N; ++i) wmg_fine<STEP>(m, U0, PackedLinks{nullptr, 0}, 0, u, w, out, P, k, key, i);
        return PT_OK;
    }
    int restrict_(const double *r, double *rc) {
        for (int t = 0; t < m.Nc * m.dc(); ++t) wmg_restrict(m, P, r, rc, t);
        return PT_OK;
    }
    int ortho() {
        for (int t = 0; t < m.Nc * 2; ++t)
            if (!wmg_ortho(m, P, t / 2, t % 2)) return PT_ERR_NUMERIC;
        return PT_OK;
    }
    int build() {
        for (int B = 0; B < m.Nc; ++B) wmg_build_site(m, U0, P, Ac, B);
        return PT_OK;
    }
    int capply(const double *v, double *out) {
        for (int B = 0; B < m.Nc; ++B) wmg_capply(m, Ac, v, out, B);
        return PT_OK;
    }
};

// ---------------------------------------------------------------- setup and solve
// near-null vectors, the prolongator and the coarse stencil
template <class X>
static int wmg_setup(X &ex, int sweeps, uint64_t seed) {
    const long n = (long)ex.m.g.N * 24;
    double *v = ex.alloc(n), *t = ex.alloc(n);
    int rc = (v && t) ? PT_OK : PT_ERR_OOM;
    for (int k = 0; k < ex.m.nv && !rc; ++k) {
        rc = ex.template fine<WMG_RANDOM>(nullptr, nullptr, v, k, pt_set_key(seed, k));
        for (int s = 0; s < sweeps && !rc; ++s)
            if (!(rc = ex.template fine<WMG_RICHARDSON>(v, nullptr, t))) rc = ex.copy(n, t, v);
        if (!rc) rc = ex.template fine<WMG_FILL>(v, nullptr, nullptr, k);
    }
    if (!rc) rc = ex.ortho();
    if (!rc) rc = ex.build();
    if (v) ex.release(v);
    if (t) ex.release(t);
    if (rc == PT_ERR_NUMERIC) pt_set_error("Wilson multigrid: a near-null vector vanished on an aggregate");
    return rc;
}

struct WMGWork {
    double *t1, *res;                                  // fine
    double *rc, *ec, *cr, *cr0, *cp, *cv, *cs, *ct;    // coarse
};

// A_c e = rc by BiCGStab from e = 0 to 1e-10 relative (at most 4 Nc dc iterations)
template <class X>
static int wmg_coarse_solve(X &ex, const WMGWork &W) {
    const long n = (long)ex.m.Nc * ex.m.dc() * 2;
    int rc;
    zd z, z2, rho, alpha;
    if ((rc = ex.zero(n, W.ec)) || (rc = ex.copy(n, W.rc, W.cr)) || (rc = ex.copy(n, W.cr, W.cr0)) ||
        (rc = ex.copy(n, W.cr, W.cp)) || (rc = ex.dot(n, 1, W.cr, W.cr, &z)))
        return rc;
    const double stop = 1e-10 * sqrt(z.re);
    rho = z;
    for (int it = 0; it < 4 * ex.m.Nc * ex.m.dc() + 20 && sqrt(z.re) > stop; ++it) {
        if ((rc = ex.capply(W.cp, W.cv)) || (rc = ex.dot(n, 1, W.cr0, W.cv, &z2))) return rc;
        alpha = zdiv(rho, z2);
        if (!std::isfinite(alpha.re) || !std::isfinite(alpha.im)) break;
        if ((rc = ex.copy(n, W.cr, W.cs)) || (rc = ex.axpy(n, 1, zd{-alpha.re, -alpha.im}, W.cv, W.cs)) ||
            (rc = ex.capply(W.cs, W.ct)) || (rc = ex.dot(n, 1, W.ct, W.ct, &z)) || (rc = ex.dot(n, 1, W.ct, W.cs, &z2)))
            return rc;
        const zd omega = z.re > 0.0 ? zd{z2.re / z.re, z2.im / z.re} : zd{0.0, 0.0};
        if ((rc = ex.axpy(n, 1, alpha, W.cp, W.ec)) || (rc = ex.axpy(n, 1, omega, W.cs, W.ec)) ||
            (rc = ex.copy(n, W.cs, W.cr)) || (rc = ex.axpy(n, 1, zd{-omega.re, -omega.im}, W.ct, W.cr)) ||
            (rc = ex.dot(n, 1, W.cr, W.cr, &z)))
            return rc;
        if (omega.re == 0.0 && omega.im == 0.0) break;
        zd rho_new;
        if ((rc = ex.dot(n, 1, W.cr0, W.cr, &rho_new))) return rc;
        const zd beta = zmulc(zdiv(rho_new, rho), zdiv(alpha, omega));
        if ((rc = ex.axpy(n, 1, zd{-omega.re, -omega.im}, W.cv, W.cp)) || (rc = ex.xpay(n, 1, W.cr, beta, W.cp)))
            return rc;
        rho = rho_new;
    }
    return PT_OK;
}

// out = M r: nu Richardson sweeps from 0, the coarse correction, nu sweeps
template <class X>
static int wmg_cycle(X &ex, int nu, const double *r, double *out, const WMGWork &W) {
    const long n = (long)ex.m.g.N * 24;
    int rc = ex.zero(n, out);
    for (int k = 0; k < nu && !rc; ++k)
        if (!(rc = ex.template fine<WMG_RICHARDSON>(out, r, W.t1))) rc = ex.copy(n, W.t1, out);
    if (!rc) rc = ex.template fine<WMG_RESIDUAL>(out, r, W.res);
    if (!rc) rc = ex.restrict_(W.res, W.rc);
    if (!rc) rc = wmg_coarse_solve(ex, W);
    if (!rc) rc = ex.template fine<WMG_PROLONG>(W.ec, nullptr, out);
    for (int k = 0; k < nu && !rc; ++k)
        if (!(rc = ex.template fine<WMG_RICHARDSON>(out, r, W.t1))) rc = ex.copy(n, W.t1, out);
    return rc;
}

// A x = b by FGMRES(mr) right-preconditioned with the cycle (Saad, Iterative
// Methods for Sparse Linear Systems, Alg. 9.6), complex Givens rotations on the
// host; x = 0 start; *relres the true relative residual at the end
template <class X>
static int wmg_fgmres(X &ex, int nu, int mr, const double *b, double *x, double tol, int maxit, int *iters,
                      double *relres) {
    const long n = (long)ex.m.g.N * 24, nc = (long)ex.m.Nc * ex.m.dc() * 2;
    std::vector<double *> V(mr + 1), Z(mr);
    for (auto &p : V) p = ex.alloc(n);
    for (auto &p : Z) p = ex.alloc(n);
    double *w = ex.alloc(n), *r = ex.alloc(n), *part = ex.alloc(2 * VEC_DOT_BLOCKS);
    WMGWork W{ex.alloc(n), ex.alloc(n), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc),
              ex.alloc(nc), ex.alloc(nc), ex.alloc(nc), ex.alloc(nc)};
    std::vector<double *> all(V);
    all.insert(all.end(), Z.begin(), Z.end());
    for (double *p : {w, r, part, W.t1, W.res, W.rc, W.ec, W.cr, W.cr0, W.cp, W.cv, W.cs, W.ct}) all.push_back(p);
    int rc = PT_OK;
    for (double *p : all)
        if (!p) rc = PT_ERR_OOM;
    if (rc) pt_set_error("Wilson multigrid solve: allocation failed");
    ex.dot_part = part;
    *iters = 0;
    *relres = 0.0;
    zd z;
    double bn = 0.0;
    bool converged = false;
    if (!rc) rc = ex.zero(n, x);
    if (!rc) rc = ex.dot(n, 1, b, b, &z);
    if (!rc) bn = sqrt(z.re);
    if (!rc && bn == 0.0) converged = true;
    std::vector<zd> H((size_t)(mr + 1) * mr), g(mr + 1), cs(mr), sn(mr), y(mr);
    while (!rc && !converged && *iters < maxit) {
        if ((rc = ex.template fine<WMG_RESIDUAL>(x, b, r)) || (rc = ex.dot(n, 1, r, r, &z))) break;
        const double beta = sqrt(z.re);
        if (beta <= tol * bn) { converged = true; break; }
        if ((rc = ex.zero(n, V[0])) || (rc = ex.axpy(n, 1, zd{1.0 / beta, 0.0}, r, V[0]))) break;
        std::fill(g.begin(), g.end(), zd{0.0, 0.0});
        g[0] = zd{beta, 0.0};
        int k = 0;
        for (int j = 0; j < mr && !rc && *iters < maxit; ++j) {
            if ((rc = wmg_cycle(ex, nu, V[j], Z[j], W)) || (rc = ex.template fine<WMG_APPLY>(Z[j], nullptr, w))) break;
            for (int i = 0; i <= j && !rc; ++i) {                       // modified Gram-Schmidt
                zd h;
                if ((rc = ex.dot(n, 1, V[i], w, &h))) break;
                H[(size_t)i * mr + j] = h;
                rc = ex.axpy(n, 1, zd{-h.re, -h.im}, V[i], w);
            }
            if (rc || (rc = ex.dot(n, 1, w, w, &z))) break;
            const double hn = sqrt(z.re);
            H[(size_t)(j + 1) * mr + j] = zd{hn, 0.0};
            for (int i = 0; i < j; ++i) {                              // earlier rotations on column j
                const zd a = H[(size_t)i * mr + j], bb = H[(size_t)(i + 1) * mr + j];
                H[(size_t)i * mr + j] = zadd(zscal(a, cs[i].re), zmulc(sn[i], bb));
                H[(size_t)(i + 1) * mr + j] = zsub(zscal(bb, cs[i].re), zmulc(zconj(sn[i]), a));
            }
            const zd a = H[(size_t)j * mr + j], bb = H[(size_t)(j + 1) * mr + j];
            const double ra = zabs(a), rr = sqrt(ra * ra + zabs(bb) * zabs(bb));
            if (rr == 0.0) { cs[j] = zd{1.0, 0.0}; sn[j] = zd{0.0, 0.0}; }
            else if (ra == 0.0) { cs[j] = zd{0.0, 0.0}; sn[j] = zd{1.0, 0.0}; }
            else {
                cs[j] = zd{ra / rr, 0.0};
                sn[j] = zscal(zmulc(zd{a.re / ra, a.im / ra}, zconj(bb)), 1.0 / rr);
            }
            H[(size_t)j * mr + j] = zadd(zscal(a, cs[j].re), zmulc(sn[j], bb));
            H[(size_t)(j + 1) * mr + j] = zd{0.0, 0.0};
            const zd gj = g[j];
            g[j] = zscal(gj, cs[j].re);
            g[j + 1] = zscal(zmulc(zconj(sn[j]), gj), -1.0);
            ++*iters;
            k = j + 1;
            if (zabs(g[j + 1]) <= tol * bn || hn == 0.0) break;
            if ((rc = ex.zero(n, V[j + 1])) || (rc = ex.axpy(n, 1, zd{1.0 / hn, 0.0}, w, V[j + 1]))) break;
        }
        if (rc) break;
        for (int i = k - 1; i >= 0; --i) {                             // R y = g
            zd s = g[i];
            for (int l = i + 1; l < k; ++l) s = zsub(s, zmulc(H[(size_t)i * mr + l], y[l]));
            y[i] = zdiv(s, H[(size_t)i * mr + i]);
        }
        for (int i = 0; i < k && !rc; ++i) rc = ex.axpy(n, 1, y[i], Z[i], x);
    }
    if (!rc && bn > 0.0) {
        if (!(rc = ex.template fine<WMG_RESIDUAL>(x, b, r)) && !(rc = ex.dot(n, 1, r, r, &z)))
            *relres = sqrt(z.re) / bn;
        if (!rc && *relres <= tol) converged = true;
    }
    for (double *p : all)
        if (p) ex.release(p);
    if (!rc && !converged) {
        pt_set_error("Wilson multigrid solve: %d iterations, relative residual %g", *iters, *relres);
        rc = PT_ERR_NOCONV;
    }
    return rc;
}

// ---------------------------------------------------------------- entry points
static int wmg_geom(const int dims[4], double kappa, int antip, int block, int nv, double omega, WMG *m,
                    const char *fn) {
    PT_CHECK_ARG(dims && block >= 1 && nv >= 1 && nv <= WMG_MAXNV && omega > 0.0 && omega <= 1.0,
                 "%s: block >= 1, 1 <= nv <= %d, 0 < omega <= 1", fn, WMG_MAXNV);
    long N = 1;
    int cs = 1;
    for (int mu = 0; mu < 4; ++mu) {
        PT_CHECK_ARG(dims[mu] >= 1 && dims[mu] % block == 0, "%s: the block side must divide every lattice side", fn);
        m->C[mu] = dims[mu] / block;
        m->cstride[mu] = cs;
        cs *= dims[mu] / block;
        N *= dims[mu];
    }
    PT_CHECK_ARG(N <= (1L << 28), "%s: lattice too large", fn);
    m->g = make_eo_geom(dims);
    m->Nc = cs;
    m->b = block;
    m->bs = block * block * block * block;
    PT_CHECK_ARG(6 * m->bs >= nv, "%s: an aggregate holds fewer components than nv", fn);
    m->nv = nv;
    m->kappa = kappa;
    m->omega = omega;
    m->o.kind = 1;
    m->o.antip = antip ? 1 : 0;
    m->o.G = make_gammas();
    m->Cb = nullptr;
    return PT_OK;
}

template <class X>
static int wmg_solve_all(X &ex, int sweeps, uint64_t seed, int nu, int restart, const double *b, double *x, int nrhs,
                         double tol, int maxit, int *iters_out, double *relres_out) {
    int rc = wmg_setup(ex, sweeps, seed), rc_nc = PT_OK;
    for (int r = 0; r < nrhs && !rc; ++r) {
        int it = 0;
        double rel = 0.0;
        const int k = wmg_fgmres(ex, nu, restart, b + (size_t)r * ex.m.g.N * 24, x + (size_t)r * ex.m.g.N * 24, tol,
                                 maxit, &it, &rel);
        if (iters_out) iters_out[r] = it;
        if (relres_out) relres_out[r] = rel;
        if (k == PT_ERR_NOCONV) rc_nc = k;
        else rc = k;
    }
    return rc ? rc : rc_nc;
}

extern "C" int pt_wmg_solve(pt_ctx *c, const pt_op *op, double csw, int block, int nv, int sweeps, int nu,
                            double omega, int restart, uint64_t seed, const double *b_dev, double *x_dev, int nrhs,
                            double tol, int maxit, int *iters_out, double *relres_out) {
    PT_CHECK_ARG(c && op && op->ctx == c && op->kind == 1, "pt_wmg_solve: a Wilson operator is required");
    PT_CHECK_ARG(nrhs >= 0 && nrhs <= 65535 && tol > 0.0 && maxit >= 1 && sweeps >= 0 && nu >= 0 && nu <= 16 &&
                     restart >= 1 && restart <= 64,
                 "pt_wmg_solve: bad nrhs, tol, maxit, sweeps, nu or restart");
    WMGDev ex;
    int rc = wmg_geom(op->dims, op->kappa, op->antip, block, nv, omega, &ex.m, "pt_wmg_solve");
    if (rc || nrhs == 0) return rc;
    PT_CHECK_ARG(b_dev && x_dev && (const double *)x_dev != b_dev, "pt_wmg_solve: NULL or aliased fields");
    PT_CUDA(cudaSetDevice(c->device));
    ex.c = c;
    ex.U1 = PackedLinks{op->U64, ex.m.g.N};
    const size_t np = (size_t)ex.m.g.N * 12 * nv * 2, na = (size_t)ex.m.Nc * 9 * ex.m.dc() * ex.m.dc() * 2;
    ex.P = ex.alloc(np);
    ex.Ac = ex.alloc(na);
    double *cb = csw != 0.0 ? ex.alloc((size_t)ex.m.g.N * 288) : nullptr;
    if (!ex.P || !ex.Ac || (csw != 0.0 && !cb)) {
        pt_set_error("pt_wmg_solve: device allocation failed");
        rc = PT_ERR_OOM;
    } else {
        if (cb) rc = pt_clover_blocks(c, op, csw, cb);
        ex.m.Cb = cb;
        if (!rc) rc = wmg_solve_all(ex, sweeps, seed, nu, restart, b_dev, x_dev, nrhs, tol, maxit, iters_out,
                                    relres_out);
    }
    if (ex.P) ex.release(ex.P);
    if (ex.Ac) ex.release(ex.Ac);
    if (cb) ex.release(cb);
    const cudaError_t ce = cudaStreamSynchronize(c->stream);
    if (!rc && ce != cudaSuccess) rc = pt_cuda_fail(ce, "pt_wmg_solve", __FILE__, __LINE__);
    return rc;
}

static int wmg_host_init(WMGHost &ex, const int dims[4], const double *U_host, double kappa, double csw, int antip,
                         int block, int nv, double omega, const char *fn) {
    PT_CHECK_ARG(U_host, "%s: NULL links", fn);
    int rc = wmg_geom(dims, kappa, antip, block, nv, omega, &ex.m, fn);
    if (rc) return rc;
    ex.U0 = UserLinks{U_host};
    ex.P = ex.alloc((size_t)ex.m.g.N * 12 * nv * 2);
    ex.Ac = ex.alloc((size_t)ex.m.Nc * 9 * ex.m.dc() * ex.m.dc() * 2);
    if (csw != 0.0) {
        double *cb = ex.alloc((size_t)ex.m.g.N * 288);
        if ((rc = pt_clover_blocks_host(dims, U_host, kappa, csw, cb))) return rc;
        ex.m.Cb = cb;
    }
    return PT_OK;
}

extern "C" int pt_wmg_solve_host(const int dims[4], const double *U_host, double kappa, double csw, int antip,
                                 int block, int nv, int sweeps, int nu, double omega, int restart, uint64_t seed,
                                 const double *b, double *x, int nrhs, double tol, int maxit, int *iters_out,
                                 double *relres_out) {
    PT_CHECK_ARG(nrhs >= 0 && b && x && tol > 0.0 && maxit >= 1 && sweeps >= 0 && nu >= 0 && nu <= 16 &&
                     restart >= 1 && restart <= 64,
                 "pt_wmg_solve_host: bad argument");
    WMGHost ex;
    int rc = wmg_host_init(ex, dims, U_host, kappa, csw, antip, block, nv, omega, "pt_wmg_solve_host");
    if (rc) return rc;
    return wmg_solve_all(ex, sweeps, seed, nu, restart, b, x, nrhs, tol, maxit, iters_out, relres_out);
}

extern "C" int pt_wmg_setup_host(const int dims[4], const double *U_host, double kappa, double csw, int antip,
                                 int block, int nv, int sweeps, double omega, uint64_t seed, double *P_out,
                                 double *Ac_out) {
    PT_CHECK_ARG(P_out && Ac_out && sweeps >= 0, "pt_wmg_setup_host: bad argument");
    WMGHost ex;
    int rc = wmg_host_init(ex, dims, U_host, kappa, csw, antip, block, nv, omega, "pt_wmg_setup_host");
    if (rc) return rc;
    if ((rc = wmg_setup(ex, sweeps, seed))) return rc;
    const size_t np = (size_t)ex.m.g.N * 12 * nv * 2, na = (size_t)ex.m.Nc * 9 * ex.m.dc() * ex.m.dc() * 2;
    std::copy(ex.P, ex.P + np, P_out);
    std::copy(ex.Ac, ex.Ac + na, Ac_out);
    return PT_OK;
}
