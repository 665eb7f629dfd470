// The Wilson-Dirac hopping term at one site, for code that runs on both the
// host and the device, with the neighbour spinors read from a user-layout
// field (full, or a half field of one parity).
#pragma once

#include "eo_geom.cuh"
#include "hd_complex.cuh"

// a field in the user layout read at a storage index: entry y of a full
// field, or entry y >> 1 of a half field
struct UserField {
    const double *f;
    int half;
    int sites;      // N or N / 2
    __host__ __device__ __forceinline__ size_t at(int y) const { return (size_t)(half ? (y >> 1) : y); }
};

struct EoOp {
    int kind;       // 0 Laplacian, 1 Wilson
    int antip;      // antiperiodic in dim 3 (Wilson)
    GammaTab G;
};

// per-site 12 x 12 blocks of one parity (entry h of a half field), e.g. the
// clover diagonal A_ee or the inverses A_oo^{-1}: out = B(h) in(site)
__host__ __device__ __forceinline__ void eo_block_site(const EoGeom &g, const double *B, int par_out,
                                                       const UserField &in, int r, int h, double *out) {
    int x[4];
    const int i = eo_full_site(g, par_out, h, x);
    const double *b = B + (size_t)h * 288, *v = in.f + ((size_t)r * in.sites + in.at(i)) * 24;
    double *o = out + ((size_t)r * g.Nh + h) * 24;
    for (int row = 0; row < 12; ++row) {
        zd acc = {0.0, 0.0};
        for (int c = 0; c < 12; ++c)
            acc = zadd(acc, zmulc(zd{b[(row * 12 + c) * 2], b[(row * 12 + c) * 2 + 1]}, zd{v[2 * c], v[2 * c + 1]}));
        o[2 * row] = acc.re;
        o[2 * row + 1] = acc.im;
    }
}

// (H psi)(x) of the Wilson hopping term at storage index i, from its
// definition: sum over mu of (1 - g_mu) U_mu(x) psi(x + mu) and
// (1 + g_mu) U_mu(x - mu)^H psi(x - mu), times -1 on the hops that cross the
// time boundary when time is antiperiodic; psi is right-hand side r of F
template <class L>
__host__ __device__ void eo_wilson_hop(const EoGeom &g, const L &U, const EoOp &o, const UserField &F, int r, int i,
                                       const int x[4], zd acc[12]) {
    for (int c = 0; c < 12; ++c) acc[c] = {0.0, 0.0};
    const double *base = F.f + (size_t)r * F.sites * 24;
    for (int mu = 0; mu < 4; ++mu)
        for (int dir = 0; dir < 2; ++dir) {
            const int y = eo_neighbour(g, i, x, mu, dir == 0 ? 1 : -1);
            const bool cross = o.antip && mu == 3 && (dir == 0 ? x[3] == g.D[3] - 1 : x[3] == 0);
            const double eta = cross ? -1.0 : 1.0;
            const double sgn = dir == 0 ? -1.0 : 1.0;         // (1 - g_mu) forward, (1 + g_mu) backward
            const double *p = base + F.at(y) * 24;
            zd chi[12];                                        // colour-rotated neighbour
            for (int s = 0; s < 4; ++s)
                for (int a = 0; a < 3; ++a) {
                    zd t = {0.0, 0.0};
                    for (int b = 0; b < 3; ++b) {
                        const zd w = dir == 0 ? U(i, mu, a * 3 + b) : zconj(U(y, mu, b * 3 + a));
                        t = zadd(t, zmulc(w, zd{p[2 * (s * 3 + b)], p[2 * (s * 3 + b) + 1]}));
                    }
                    chi[s * 3 + a] = t;
                }
            for (int s = 0; s < 4; ++s)
                for (int a = 0; a < 3; ++a) {
                    zd gchi = {0.0, 0.0};
                    for (int t = 0; t < 4; ++t) gchi = zadd(gchi, zmulc(o.G.g[mu][s * 4 + t], chi[t * 3 + a]));
                    acc[s * 3 + a] = zadd(acc[s * 3 + a], zscal(zadd(chi[s * 3 + a], zscal(gchi, sgn)), eta));
                }
        }
}

