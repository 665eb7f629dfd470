/*
 * Oracle (test infrastructure only): greedy displaced distance-k colouring.
 *
 * Algorithm 1 (Sec. 3.1): visit the lattice nodes in a given order; each node
 * receives the smallest colour not already held by a node of its displaced
 * neighbourhood N(x,p,k) (given as a stencil of coordinate offsets, Eq. (8),
 * Algorithm 2).  Nodes not yet visited hold no colour.  Colours are 0-based
 * here (the paper counts from 1).  A used-colour table of |stencil|+1 entries
 * suffices because a node has at most |stencil| neighbours (Sec. 3.1).
 *
 * Plain, sequential C: no blocking or reordering.  Built by oracle/build.py.
 */
#include <stdint.h>
#include <stdlib.h>

int oracle_greedy_colour(int d, const int *dims, int n_off, const int *offsets,
                         const int64_t *visit, int32_t *col)
{
    int64_t N = 1;
    for (int mu = 0; mu < d; ++mu) N *= dims[mu];
    for (int64_t i = 0; i < N; ++i) col[i] = -1;

    /* each offset reduced once to [0, D_mu) per dimension, so that the
     * neighbour's coordinate needs at most one subtraction of D_mu */
    int *red = (int *)malloc(sizeof(int) * (size_t)(n_off > 0 ? n_off : 1) * (size_t)d);
    /* used[c] == stamp  <=>  colour c is taken in the current neighbourhood */
    int64_t *used = (int64_t *)calloc((size_t)n_off + 2, sizeof(int64_t));
    if (!used || !red) { free(used); free(red); return -1; }
    for (int o = 0; o < n_off; ++o)
        for (int mu = 0; mu < d; ++mu) {
            int c = offsets[o * d + mu] % dims[mu];
            red[o * d + mu] = c < 0 ? c + dims[mu] : c;
        }
    int n_colours = 0;
    int x[8];
    for (int64_t t = 0; t < N; ++t) {
        int64_t site = visit[t];
        int64_t stamp = t + 1;
        int64_t rem = site;
        for (int mu = 0; mu < d; ++mu) { x[mu] = (int)(rem % dims[mu]); rem /= dims[mu]; }
        for (int o = 0; o < n_off; ++o) {
            int64_t idx = 0, stride = 1;
            for (int mu = 0; mu < d; ++mu) {
                int c = x[mu] + red[o * d + mu];
                if (c >= dims[mu]) c -= dims[mu];
                idx += (int64_t)c * stride;
                stride *= dims[mu];
            }
            if (idx == site) continue;          /* x is excluded from N(x,p,k) */
            int32_t cy = col[idx];
            if (cy >= 0 && cy <= n_off) used[cy] = stamp;
        }
        int c = 0;
        while (used[c] == stamp) ++c;
        col[site] = c;
        if (c + 1 > n_colours) n_colours = c + 1;
    }
    free(red);
    free(used);
    return n_colours;
}

/*
 * Nested variant (the hierarchical reading of a colouring grown from k1 to
 * k2 > k1): the same walk, but a node only sees the neighbours that share its
 * parent colour parent[] (the k1 colouring).  The colours returned are local
 * to each parent class; the caller pairs them with the parent colour.
 */
int oracle_greedy_colour_nested(int d, const int *dims, int n_off, const int *offsets, const int64_t *visit,
                                const int32_t *parent, int32_t *col)
{
    int64_t N = 1;
    for (int mu = 0; mu < d; ++mu) N *= dims[mu];
    for (int64_t i = 0; i < N; ++i) col[i] = -1;
    int64_t *used = (int64_t *)calloc((size_t)n_off + 2, sizeof(int64_t));
    if (!used) return -1;
    int n_colours = 0;
    int x[8];
    for (int64_t t = 0; t < N; ++t) {
        int64_t site = visit[t];
        int64_t stamp = t + 1;
        int64_t rem = site;
        for (int mu = 0; mu < d; ++mu) { x[mu] = (int)(rem % dims[mu]); rem /= dims[mu]; }
        for (int o = 0; o < n_off; ++o) {
            int64_t idx = 0, stride = 1;
            for (int mu = 0; mu < d; ++mu) {
                int c = (x[mu] + offsets[o * d + mu]) % dims[mu];
                if (c < 0) c += dims[mu];
                idx += (int64_t)c * stride;
                stride *= dims[mu];
            }
            if (idx == site || parent[idx] != parent[site]) continue;
            int32_t cy = col[idx];
            if (cy >= 0 && cy <= n_off) used[cy] = stamp;
        }
        int c = 0;
        while (used[c] == stamp) ++c;
        col[site] = c;
        if (c + 1 > n_colours) n_colours = c + 1;
    }
    free(used);
    return n_colours;
}
