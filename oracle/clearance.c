/*
 * Oracle (test infrastructure only): colour coincidences at fixed offsets.
 *
 * For each offset o (a vector of d integers, any sign), count the nodes x of
 * the torus whose colour equals that of x + o (mod D).  The clearance
 * statistic of Sec. 4.3 (Table 5) is a sum of these counts over the offsets
 * of a shell, divided by the shell size and the number of nodes.
 *
 * Plain C: a loop over offsets, nested loops over the nodes' coordinates.
 * Lattices of up to four dimensions.  Built by oracle/build.py.
 */
#include <stdint.h>

void oracle_offset_matches(int d, const int *dims, const int32_t *col, int n_off, const int *offsets,
                           int64_t *matches)
{
    /* the lattice as four dimensions (missing ones of length 1), first fastest */
    int D[4] = {1, 1, 1, 1};
    for (int mu = 0; mu < d && mu < 4; ++mu) D[mu] = dims[mu];
    const int64_t s1 = D[0], s2 = (int64_t)D[0] * D[1], s3 = (int64_t)D[0] * D[1] * D[2];
    for (int o = 0; o < n_off; ++o) {
        int r[4] = {0, 0, 0, 0};                   /* the offset reduced to [0, D_mu) */
        for (int mu = 0; mu < d && mu < 4; ++mu) {
            int c = offsets[o * d + mu] % D[mu];
            r[mu] = c < 0 ? c + D[mu] : c;
        }
        int64_t count = 0;
        for (int x3 = 0; x3 < D[3]; ++x3) {
            int y3 = x3 + r[3] < D[3] ? x3 + r[3] : x3 + r[3] - D[3];
            for (int x2 = 0; x2 < D[2]; ++x2) {
                int y2 = x2 + r[2] < D[2] ? x2 + r[2] : x2 + r[2] - D[2];
                for (int x1 = 0; x1 < D[1]; ++x1) {
                    int y1 = x1 + r[1] < D[1] ? x1 + r[1] : x1 + r[1] - D[1];
                    const int32_t *cx = col + x1 * s1 + x2 * s2 + x3 * s3;    /* the row of x */
                    const int32_t *cy = col + y1 * s1 + y2 * s2 + y3 * s3;    /* the row of x + o */
                    /* along the first dimension x0 + r0 wraps once, at x0 = D0 - r0 */
                    for (int x0 = 0; x0 < D[0] - r[0]; ++x0) count += cx[x0] == cy[x0 + r[0]];
                    for (int x0 = D[0] - r[0]; x0 < D[0]; ++x0) count += cx[x0] == cy[x0 + r[0] - D[0]];
                }
            }
        }
        matches[o] = count;
    }
}
