/*
 * lbm_oracle.c -- plain FP64 CPU oracle for the pore-scale lattice Boltzmann
 * method of Fattahi, Waluga, Wohlmuth & Ruede, "Large scale lattice Boltzmann
 * simulation for the coupling of free and porous media flow" (Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library; the two are compared on the
 * same seeded inputs.
 *
 * What it computes, in the order the paper states it:
 *   - D3Q19 populations f_k(x,t), k = 0..18 (Sec. 2.1, Eq. (LBM)).
 *   - TRT collision: symmetric/antisymmetric split (Eq. (TRT2)) relaxed with
 *     omega+ and omega- (Eq. (TRT)); 1/omega+ = 3 nu + 1/2 and the magic
 *     parameter Lambda = (1/omega+ - 1/2)(1/omega- - 1/2) fixes omega-.
 *   - Incompressible equilibrium with rho0 = 1, c_s^2 = 1/3
 *     (Eq. (equilibrium)); density and momentum are the zeroth and first
 *     moments (Eq. (Macro)).
 *   - Body-force source F_k added to the post-collision state
 *     (Eq. (collision)), then streaming (Eq. (streaming)) into a second
 *     array ("dense, two-array, collide then stream").
 *   - Walls: central linear interpolation (Eq. (CLI)) on every link from a
 *     fluid node to a solid node, with q the fraction of the link that lies in
 *     the fluid; q = 1/2 is simple bounce-back (Eq. (noslip)).
 *   - Post-processing: plane averages of the stream-wise velocity (Sec. 3.1)
 *     and Darcy permeability (Eq. (Darcy)).
 *
 * Readings of points the paper leaves open (each one is restated where it is
 * used): velocity ordering and weights of D3Q19; the source term
 * F_k = 3 w_k e_k.g added after relaxation with the equilibrium built from the
 * pre-collision momentum j, and the reported velocity u = j + g/2; full
 * (unshifted) populations with rho = sum f; the second fluid node of a link is
 * x_f2 = x_f1 - e_k, and the link falls back to bounce-back when x_f2 is solid
 * (Eq. (CLI) has no second node there); optionally (the "safeguards", off by
 * default) also when x_f1 - 2 e_k is solid or when q < 0.1, which stabilises
 * sharp corners of overlapping packings (see orc_link_fallback);
 * q is the first point of the link on a solid surface (smallest entry
 * parameter);
 * seeded sphere placement (SplitMix64) stands in for the rigid-body packing.
 *
 * Plain loops, no blocking or fusion beyond the definition; OpenMP only splits
 * independent per-cell loops and never changes an arithmetic order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define NQ 19

/* D3Q19 (Sec. 2.1): rest; +-x, +-y, +-z; then the twelve face diagonals in
 * opposite pairs, so that the opposite of k is k+1 for odd k and k-1 for even
 * k.  The paper prints no ordering; this one is a convention of this project. */
static const int ORC_EX[NQ] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int ORC_EY[NQ] = {0, 0, 0, 1, -1, 0, 0, 1, -1, -1, 1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int ORC_EZ[NQ] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, -1, -1, 1, 1, -1, -1, 1};

/* Standard D3Q19 weights, normalised to unity (Eq. (equilibrium)). */
static double orc_weight(int k)
{
    if (k == 0) return 1.0 / 3.0;
    if (k <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

static int orc_opp(int k)
{
    if (k == 0) return 0;
    return (k & 1) ? k + 1 : k - 1;
}

void orc_velocity_set(int32_t *e /* [19][3] */, double *w /* [19] */)
{
    for (int k = 0; k < NQ; ++k) {
        e[3 * k + 0] = ORC_EX[k];
        e[3 * k + 1] = ORC_EY[k];
        e[3 * k + 2] = ORC_EZ[k];
        w[k] = orc_weight(k);
    }
}

int orc_opposite(int k) { return orc_opp(k); }

/* ------------------------------------------------------------------------- */
/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): a Weyl sequence with step  */
/* 0x9e3779b97f4a7c15 passed through a 64-bit finaliser.                     */
/* ------------------------------------------------------------------------- */
uint64_t orc_splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state += 0x9e3779b97f4a7c15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Uniform double in [0,1) from the top 53 bits. */
double orc_uniform(uint64_t *state)
{
    return (double)(orc_splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0);
}

/* Sphere data are kept on the 2^-10 grid so that every voxel test and every
 * link fraction below is exact or correctly rounded in FP64. */
static double orc_quantize(double v) { return floor(v * 1024.0) / 1024.0; }

/* ------------------------------------------------------------------------- */
/* Box: x and y are periodic.  z is periodic, or bounded by the solid wall    */
/* layers z = 0 and z = nz-1 whose surfaces lie at the link fractions q_lo    */
/* and q_hi from the adjacent fluid nodes (1/2: half-way, Eq. (noslip)).      */
/* ------------------------------------------------------------------------- */
typedef struct {
    int nx, ny, nz, periodic_z;
    double q_lo, q_hi;
} orc_box;

static int64_t orc_cell(const orc_box *b, int x, int y, int z)
{
    return (int64_t)x + (int64_t)b->nx * ((int64_t)y + (int64_t)b->ny * (int64_t)z);
}

static int orc_wrap(int v, int n)
{
    if (v < 0) return v + n;
    if (v >= n) return v - n;
    return v;
}

static int orc_is_wall_layer(const orc_box *b, int z)
{
    return !b->periodic_z && (z == 0 || z == b->nz - 1);
}

/* Stamp one sphere (all periodic images) into the solid mask.  Returns the
 * number of cells with layer_lo <= z < layer_hi (outside wall layers) that
 * turned from fluid to solid. */
static int64_t orc_stamp_sphere(const orc_box *b, uint8_t *solid, double cx, double cy, double cz,
                                double r, int layer_lo, int layer_hi)
{
    int64_t newly = 0;
    int mz_lo = b->periodic_z ? -1 : 0, mz_hi = b->periodic_z ? 1 : 0;
    for (int mx = -1; mx <= 1; ++mx)
        for (int my = -1; my <= 1; ++my)
            for (int mz = mz_lo; mz <= mz_hi; ++mz) {
                double ix = cx + mx * b->nx, iy = cy + my * b->ny, iz = cz + mz * b->nz;
                int x0 = (int)ceil(ix - r), x1 = (int)floor(ix + r);
                int y0 = (int)ceil(iy - r), y1 = (int)floor(iy + r);
                int z0 = (int)ceil(iz - r), z1 = (int)floor(iz + r);
                if (x0 < 0) x0 = 0;
                if (y0 < 0) y0 = 0;
                if (z0 < 0) z0 = 0;
                if (x1 > b->nx - 1) x1 = b->nx - 1;
                if (y1 > b->ny - 1) y1 = b->ny - 1;
                if (z1 > b->nz - 1) z1 = b->nz - 1;
                for (int z = z0; z <= z1; ++z)
                    for (int y = y0; y <= y1; ++y)
                        for (int x = x0; x <= x1; ++x) {
                            double dx = x - ix, dy = y - iy, dz = z - iz;
                            if (dx * dx + dy * dy + dz * dz <= r * r) {
                                int64_t c = orc_cell(b, x, y, z);
                                if (!solid[c]) {
                                    solid[c] = 1;
                                    if (z >= layer_lo && z < layer_hi && !orc_is_wall_layer(b, z)) ++newly;
                                }
                            }
                        }
            }
    return newly;
}

static void orc_wall_layers(const orc_box *b, uint8_t *solid)
{
    if (b->periodic_z) return;
    for (int y = 0; y < b->ny; ++y)
        for (int x = 0; x < b->nx; ++x) {
            solid[orc_cell(b, x, y, 0)] = 1;
            solid[orc_cell(b, x, y, b->nz - 1)] = 1;
        }
}

/* Solid mask: a cell (integer centre) is solid when it lies in a wall layer or
 * inside (distance <= r) any periodic image of any sphere (Sec. 3.1: the sphere
 * geometry defines the solid matrix and is resolved by the lattice). */
void orc_voxelize(int nx, int ny, int nz, int periodic_z, const double *xyzr, int64_t n,
                  uint8_t *solid)
{
    orc_box b = {nx, ny, nz, periodic_z, 0.5, 0.5};
    memset(solid, 0, (size_t)nx * ny * nz);
    orc_wall_layers(&b, solid);
    for (int64_t s = 0; s < n; ++s)
        orc_stamp_sphere(&b, solid, xyzr[4 * s], xyzr[4 * s + 1], xyzr[4 * s + 2], xyzr[4 * s + 3], 0, 0);
}

/* Seeded sphere placement standing in for the settled rigid-body packing of
 * Sec. 3.1.  Each candidate draws, in this order, its centre x in [0,nx), y in
 * [0,ny), z in [z0,z1) and its radius in [r_min,r_max), each quantised down to
 * the 2^-10 grid.  Without overlap, a candidate whose minimum-image centre
 * distance to an earlier sphere is below the radius sum is rejected; after
 * max_rejects consecutive rejections the packing fails (-2).  Spheres are added
 * until the voxel porosity of the cells with ceil(z0) <= z < ceil(z1) (outside
 * wall layers) is at most the target.  Returns 0, -1 (bad arguments or more
 * than max_spheres needed) or -2. */
int orc_place_spheres(int nx, int ny, int nz, int periodic_z, double z0, double z1, double r_min,
                      double r_max, double porosity, int allow_overlap, uint64_t seed,
                      int64_t max_spheres, int64_t max_rejects, double *xyzr, int64_t *n_out,
                      double *porosity_out)
{
    orc_box b = {nx, ny, nz, periodic_z, 0.5, 0.5};
    if (nx <= 0 || ny <= 0 || nz <= 0 || !(z1 > z0) || !(r_max >= r_min) || !(r_min > 0.0))
        return -1;
    if (2.0 * r_max >= nx || 2.0 * r_max >= ny || (periodic_z && 2.0 * r_max >= nz)) return -1;
    uint8_t *solid = (uint8_t *)calloc((size_t)nx * ny * nz, 1);
    if (!solid) return -1;
    orc_wall_layers(&b, solid);
    int layer_lo = (int)ceil(z0), layer_hi = (int)ceil(z1);
    int64_t layer_cells = 0, layer_fluid;
    for (int z = layer_lo; z < layer_hi; ++z)
        if (z >= 0 && z < nz && !orc_is_wall_layer(&b, z)) layer_cells += (int64_t)nx * ny;
    layer_fluid = layer_cells;
    uint64_t state = seed;
    int64_t n = 0, rejects = 0;
    int rc = 0;
    double phi = layer_cells ? 1.0 : 0.0;
    while (layer_cells > 0 && phi > porosity) {
        double cx = orc_quantize(orc_uniform(&state) * nx);
        double cy = orc_quantize(orc_uniform(&state) * ny);
        double cz = orc_quantize(z0 + orc_uniform(&state) * (z1 - z0));
        double r = orc_quantize(r_min + orc_uniform(&state) * (r_max - r_min));
        if (!allow_overlap) {
            int clash = 0;
            for (int64_t j = 0; j < n && !clash; ++j) {
                double dx = cx - xyzr[4 * j], dy = cy - xyzr[4 * j + 1], dz = cz - xyzr[4 * j + 2];
                if (dx > 0.5 * nx) dx -= nx;
                if (dx < -0.5 * nx) dx += nx;
                if (dy > 0.5 * ny) dy -= ny;
                if (dy < -0.5 * ny) dy += ny;
                if (periodic_z) {
                    if (dz > 0.5 * nz) dz -= nz;
                    if (dz < -0.5 * nz) dz += nz;
                }
                double rs = r + xyzr[4 * j + 3];
                if (dx * dx + dy * dy + dz * dz < rs * rs) clash = 1;
            }
            if (clash) {
                if (++rejects >= max_rejects) { rc = -2; break; }
                continue;
            }
        }
        rejects = 0;
        if (n >= max_spheres) { rc = -1; break; }
        xyzr[4 * n] = cx;
        xyzr[4 * n + 1] = cy;
        xyzr[4 * n + 2] = cz;
        xyzr[4 * n + 3] = r;
        ++n;
        layer_fluid -= orc_stamp_sphere(&b, solid, cx, cy, cz, r, layer_lo, layer_hi);
        phi = (double)layer_fluid / (double)layer_cells;
    }
    free(solid);
    *n_out = n;
    *porosity_out = phi;
    return rc;
}

/* ------------------------------------------------------------------------- */
/* Link fraction q (Eq. (CLI)): q = |x_f1 - x_w| / |x_f1 - x_b| where x_w is  */
/* the first point of the link from the fluid node x_f1 to the solid node     */
/* x_b = x_f1 + e_k that lies on a solid surface.  Candidates are the entry   */
/* parameter s in (0,1] of every sphere image the link enters and, when x_b   */
/* lies in a wall layer, that wall's q.  q is the smallest candidate.         */
/* ------------------------------------------------------------------------- */

/* Smaller root of A s^2 + 2 B s + C = 0 for the ray x + s e against the sphere
 * |p - c| <= r, d = x - c (x outside, so C > 0).  Returns 2 (no candidate)
 * unless the ray approaches the sphere (B < 0), meets it (B^2 - A C >= 0) and
 * enters it within the link (s <= 1). */
static double orc_sphere_entry(double dx, double dy, double dz, int ex, int ey, int ez, double r)
{
    double A = (double)(ex * ex + ey * ey + ez * ez);
    double B = dx * ex + dy * ey + dz * ez;
    double C = dx * dx + dy * dy + dz * dz - r * r;
    double disc = B * B - A * C;
    if (!(B < 0.0) || disc < 0.0) return 2.0;
    double s = (-B - sqrt(disc)) / A;
    return s <= 1.0 ? s : 2.0;
}

/* One sphere image: sphere index and periodic shift. */
typedef struct {
    int32_t s;
    int8_t mx, my, mz;
} orc_image;

static double orc_wall_candidate(const orc_box *b, int bz)
{
    double q = 2.0;
    if (!b->periodic_z) {
        if (bz <= 0) q = b->q_lo;
        if (bz >= b->nz - 1 && b->q_hi < q) q = b->q_hi;
    }
    return q;
}

static double orc_image_candidate(const orc_box *b, const double *xyzr, orc_image im, int x, int y,
                                  int z, int k)
{
    double cx = xyzr[4 * im.s] + im.mx * b->nx;
    double cy = xyzr[4 * im.s + 1] + im.my * b->ny;
    double cz = xyzr[4 * im.s + 2] + im.mz * b->nz;
    return orc_sphere_entry(x - cx, y - cy, z - cz, ORC_EX[k], ORC_EY[k], ORC_EZ[k], xyzr[4 * im.s + 3]);
}

/* q by testing every image of every sphere. */
static double orc_link_q_impl(const orc_box *b, const double *xyzr, int64_t n, int x, int y, int z,
                              int k)
{
    double q = orc_wall_candidate(b, z + ORC_EZ[k]);
    int mz_lo = b->periodic_z ? -1 : 0, mz_hi = b->periodic_z ? 1 : 0;
    for (int64_t s = 0; s < n; ++s)
        for (int mx = -1; mx <= 1; ++mx)
            for (int my = -1; my <= 1; ++my)
                for (int mz = mz_lo; mz <= mz_hi; ++mz) {
                    orc_image im = {(int32_t)s, (int8_t)mx, (int8_t)my, (int8_t)mz};
                    double sv = orc_image_candidate(b, xyzr, im, x, y, z, k);
                    if (sv < q) q = sv;
                }
    return q;
}

/* q of one link, for hand-made cases: spheres as [n][4] (x,y,z,r). */
double orc_link_q(int nx, int ny, int nz, int periodic_z, double q_lo, double q_hi,
                  const double *xyzr, int64_t n, int x, int y, int z, int k)
{
    orc_box b = {nx, ny, nz, periodic_z, q_lo, q_hi};
    return orc_link_q_impl(&b, xyzr, n, x, y, z, k);
}

/* Pruning for large boxes: the box is cut into bins of ORC_BIN^3 cells and
 * every sphere image is listed in each bin that its bounding box, grown by two
 * cells, overlaps.  A link from x_f1 can only enter images listed in the bin
 * of x_f1 (the link is at most sqrt(2) long), so the minimum over that list
 * equals the minimum over all images. */
#define ORC_BIN 8
typedef struct {
    int nbx, nby, nbz;
    int64_t *start; /* [nbins+1] */
    orc_image *img;
} orc_bins;

static void orc_bins_free(orc_bins *bs)
{
    free(bs->start);
    free(bs->img);
}

static int orc_bins_build(const orc_box *b, const double *xyzr, int64_t n, orc_bins *bs)
{
    bs->nbx = (b->nx + ORC_BIN - 1) / ORC_BIN;
    bs->nby = (b->ny + ORC_BIN - 1) / ORC_BIN;
    bs->nbz = (b->nz + ORC_BIN - 1) / ORC_BIN;
    int64_t nb = (int64_t)bs->nbx * bs->nby * bs->nbz;
    bs->start = (int64_t *)calloc((size_t)nb + 1, sizeof(int64_t));
    bs->img = NULL;
    if (!bs->start) return -1;
    int mz_lo = b->periodic_z ? -1 : 0, mz_hi = b->periodic_z ? 1 : 0;
    for (int pass = 0; pass < 2; ++pass) {
        int64_t *fill = NULL;
        if (pass == 1) {
            for (int64_t i = 0; i < nb; ++i) bs->start[i + 1] += bs->start[i];
            bs->img = (orc_image *)malloc(sizeof(orc_image) * (size_t)(bs->start[nb] ? bs->start[nb] : 1));
            fill = (int64_t *)malloc(sizeof(int64_t) * (size_t)nb);
            if (!bs->img || !fill) { free(fill); return -1; }
            memcpy(fill, bs->start, sizeof(int64_t) * (size_t)nb);
        }
        for (int64_t s = 0; s < n; ++s)
            for (int mx = -1; mx <= 1; ++mx)
                for (int my = -1; my <= 1; ++my)
                    for (int mz = mz_lo; mz <= mz_hi; ++mz) {
                        double r = xyzr[4 * s + 3] + 2.0;
                        double cx = xyzr[4 * s] + mx * b->nx, cy = xyzr[4 * s + 1] + my * b->ny;
                        double cz = xyzr[4 * s + 2] + mz * b->nz;
                        int lo[3] = {(int)floor(cx - r), (int)floor(cy - r), (int)floor(cz - r)};
                        int hi[3] = {(int)ceil(cx + r), (int)ceil(cy + r), (int)ceil(cz + r)};
                        int dims[3] = {b->nx, b->ny, b->nz};
                        int skip = 0;
                        for (int d = 0; d < 3; ++d) {
                            if (lo[d] < 0) lo[d] = 0;
                            if (hi[d] > dims[d] - 1) hi[d] = dims[d] - 1;
                            if (lo[d] > hi[d]) skip = 1;
                        }
                        if (skip) continue;
                        orc_image im = {(int32_t)s, (int8_t)mx, (int8_t)my, (int8_t)mz};
                        for (int bz = lo[2] / ORC_BIN; bz <= hi[2] / ORC_BIN; ++bz)
                            for (int by = lo[1] / ORC_BIN; by <= hi[1] / ORC_BIN; ++by)
                                for (int bx = lo[0] / ORC_BIN; bx <= hi[0] / ORC_BIN; ++bx) {
                                    int64_t bi = bx + (int64_t)bs->nbx * (by + (int64_t)bs->nby * bz);
                                    if (pass == 0) ++bs->start[bi + 1];
                                    else bs->img[fill[bi]++] = im;
                                }
                    }
        free(fill);
    }
    return 0;
}

static double orc_link_q_binned(const orc_box *b, const double *xyzr, const orc_bins *bs, int x,
                                int y, int z, int k)
{
    double q = orc_wall_candidate(b, z + ORC_EZ[k]);
    int64_t bi = x / ORC_BIN + (int64_t)bs->nbx * (y / ORC_BIN + (int64_t)bs->nby * (z / ORC_BIN));
    for (int64_t i = bs->start[bi]; i < bs->start[bi + 1]; ++i) {
        double sv = orc_image_candidate(b, xyzr, bs->img[i], x, y, z, k);
        if (sv < q) q = sv;
    }
    return q;
}

/* Neighbour cell of (x,y,z) along e_k; -1 when it leaves the box through a
 * non-periodic face (the region beyond counts as wall). */
static int64_t orc_neighbour(const orc_box *b, int x, int y, int z, int k)
{
    int xn = orc_wrap(x + ORC_EX[k], b->nx), yn = orc_wrap(y + ORC_EY[k], b->ny);
    int zn = z + ORC_EZ[k];
    if (b->periodic_z) zn = orc_wrap(zn, b->nz);
    else if (zn < 0 || zn >= b->nz) return -1;
    return orc_cell(b, xn, yn, zn);
}

/* Bounce-back fallback of link (x, k) with fraction q.  Eq. (CLI) needs the
 * second fluid node x_f2 = x_f1 - e_k, so the link uses simple bounce-back
 * (a = 0) when x_f2 is solid: this is the only fallback of the paper's scheme.
 * With `safeguards` set, two more cases take bounce-back because the FP64
 * update was observed to grow without bound there, in the sharp corners of
 * overlapping sphere packings (nodes with most of their 18 links cut):
 *   - x_f2 is itself a wall node on the link's line (x_f1 - 2 e_k solid: a
 *     two-cell gap, where the two interpolations feed each other);
 *   - q < ORC_CLI_QMIN: the wall within a tenth of a link of the node, where
 *     a = (1-2q)/(1+2q) > 2/3 weights the non-local term almost fully.
 * Either case alone left some corners unstable; together they stabilised
 * every one found. */
#define ORC_CLI_QMIN 0.1
static int orc_link_fallback(const orc_box *b, const uint8_t *solid, int x, int y, int z, int k, double q,
                             int safeguards)
{
    const int kb = orc_opp(k);
    int64_t c2 = orc_neighbour(b, x, y, z, kb);
    if (c2 < 0 || solid[c2]) return 1;
    if (!safeguards) return 0;
    if (q < ORC_CLI_QMIN) return 1;
    int x2 = orc_wrap(x + ORC_EX[kb], b->nx), y2 = orc_wrap(y + ORC_EY[kb], b->ny), z2 = z + ORC_EZ[kb];
    if (b->periodic_z) z2 = orc_wrap(z2, b->nz);
    int64_t c3 = orc_neighbour(b, x2, y2, z2, kb);
    return c3 < 0 || solid[c3];
}

/* ------------------------------------------------------------------------- */
/* Fluid list, neighbour table and wall-link list.                            */
/* fluid_cell[i]  : linear cell index (x fastest) of the i-th fluid cell, in  */
/*                  increasing cell order.                                    */
/* nbr[(k-1)*nf+i]: fluid index of the neighbour along e_k, -1 when solid.    */
/* links          : one record per (fluid cell, k) with a solid neighbour,   */
/*                  sorted by (cell, k): cell index i, k, q, and whether the  */
/*                  link falls back to bounce-back (orc_link_fallback, with   */
/*                  the corner safeguards when `safeguards` is set).          */
/* Call with fluid_cell == NULL to get counts only.                           */
/* ------------------------------------------------------------------------- */
int orc_build_lists(int nx, int ny, int nz, int periodic_z, double q_lo, double q_hi,
                    const double *xyzr, int64_t n, int64_t *nf_out, int64_t *nlinks_out,
                    int32_t *fluid_cell, int32_t *nbr, int32_t *link_cell, int8_t *link_k,
                    double *link_q, uint8_t *link_fallback, int use_bins, int safeguards)
{
    orc_box b = {nx, ny, nz, periodic_z, q_lo, q_hi};
    int64_t ncell = (int64_t)nx * ny * nz;
    uint8_t *solid = (uint8_t *)malloc((size_t)ncell);
    int32_t *index = (int32_t *)malloc(sizeof(int32_t) * (size_t)ncell);
    orc_bins bins = {0, 0, 0, NULL, NULL};
    if (!solid || !index || (use_bins && orc_bins_build(&b, xyzr, n, &bins) != 0)) {
        free(solid); free(index); orc_bins_free(&bins); return -1;
    }
    orc_voxelize(nx, ny, nz, periodic_z, xyzr, n, solid);
    int64_t nf = 0;
    for (int64_t c = 0; c < ncell; ++c) index[c] = solid[c] ? -1 : (int32_t)nf++;
    int64_t nl = 0;
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = orc_cell(&b, x, y, z);
                if (solid[c]) continue;
                int32_t i = index[c];
                if (fluid_cell) fluid_cell[i] = (int32_t)c;
                for (int k = 1; k < NQ; ++k) {
                    int64_t cn = orc_neighbour(&b, x, y, z, k);
                    int32_t in = (cn >= 0 && !solid[cn]) ? index[cn] : -1;
                    if (nbr) nbr[(int64_t)(k - 1) * nf + i] = in;
                    if (in >= 0) continue;
                    if (link_cell) {
                        link_cell[nl] = i;
                        link_k[nl] = (int8_t)k;
                        link_q[nl] = use_bins ? orc_link_q_binned(&b, xyzr, &bins, x, y, z, k)
                                              : orc_link_q_impl(&b, xyzr, n, x, y, z, k);
                        link_fallback[nl] = (uint8_t)orc_link_fallback(&b, solid, x, y, z, k, link_q[nl], safeguards);
                    }
                    ++nl;
                }
            }
    *nf_out = nf;
    *nlinks_out = nl;
    free(solid);
    free(index);
    orc_bins_free(&bins);
    return 0;
}

/* ------------------------------------------------------------------------- */
/* The LBM itself.                                                            */
/* ------------------------------------------------------------------------- */
typedef struct orc_lbm {
    orc_box b;
    int64_t ncell;
    uint8_t *solid;
    double *f;     /* [19][ncell]: populations f_k(x, t_n); collided in place */
    double *fn;    /* [19][ncell]: streamed populations f_k(x, t_{n+1})        */
    double *uprev; /* [3][ncell]: velocity snapshot for the residual            */
    int has_prev;
    /* wall links, grouped per cell: link_start[c]..link_start[c+1] */
    int64_t *link_start;
    int8_t *link_k;
    double *link_a; /* (1-2q)/(1+2q); 0 for the bounce-back fallback */
    double omega_p, omega_m, nu;
    double g[3];
    int64_t steps;
} orc_lbm;

void orc_lbm_destroy(orc_lbm *s)
{
    if (!s) return;
    free(s->solid);
    free(s->f);
    free(s->fn);
    free(s->uprev);
    free(s->link_start);
    free(s->link_k);
    free(s->link_a);
    free(s);
}

/* Relaxation rates (Sec. 2.1): 1/omega+ = 3 nu + 1/2 with tau = 1/omega+;
 * omega- from the magic parameter Lambda = (1/omega+ - 1/2)(1/omega- - 1/2). */
void orc_rates(double tau, double lambda, double *omega_p, double *omega_m, double *nu)
{
    *omega_p = 1.0 / tau;
    *nu = (tau - 0.5) / 3.0;
    *omega_m = 1.0 / (lambda / (tau - 0.5) + 0.5);
}

orc_lbm *orc_lbm_create(int nx, int ny, int nz, int periodic_z, double q_lo, double q_hi,
                        const double *xyzr, int64_t n, double tau, double lambda, double gx,
                        double gy, double gz, int safeguards)
{
    orc_lbm *s = (orc_lbm *)calloc(1, sizeof(orc_lbm));
    if (!s) return NULL;
    s->b = (orc_box){nx, ny, nz, periodic_z, q_lo, q_hi};
    s->ncell = (int64_t)nx * ny * nz;
    s->solid = (uint8_t *)malloc((size_t)s->ncell);
    s->f = (double *)calloc((size_t)NQ * s->ncell, sizeof(double));
    s->fn = (double *)calloc((size_t)NQ * s->ncell, sizeof(double));
    s->uprev = (double *)calloc((size_t)3 * s->ncell, sizeof(double));
    s->link_start = (int64_t *)calloc((size_t)s->ncell + 1, sizeof(int64_t));
    if (!s->solid || !s->f || !s->fn || !s->uprev || !s->link_start) { orc_lbm_destroy(s); return NULL; }
    orc_voxelize(nx, ny, nz, periodic_z, xyzr, n, s->solid);
    /* count links per cell, then fill */
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = orc_cell(&s->b, x, y, z), cnt = 0;
                if (!s->solid[c])
                    for (int k = 1; k < NQ; ++k) {
                        int64_t cn = orc_neighbour(&s->b, x, y, z, k);
                        if (cn < 0 || s->solid[cn]) ++cnt;
                    }
                s->link_start[c + 1] = cnt;
            }
    for (int64_t c = 0; c < s->ncell; ++c) s->link_start[c + 1] += s->link_start[c];
    int64_t nl = s->link_start[s->ncell];
    s->link_k = (int8_t *)malloc((size_t)(nl ? nl : 1));
    s->link_a = (double *)malloc(sizeof(double) * (size_t)(nl ? nl : 1));
    if (!s->link_k || !s->link_a) { orc_lbm_destroy(s); return NULL; }
    orc_bins bins;
    if (orc_bins_build(&s->b, xyzr, n, &bins) != 0) { orc_bins_free(&bins); orc_lbm_destroy(s); return NULL; }
#pragma omp parallel for schedule(dynamic, 1)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int64_t c = orc_cell(&s->b, x, y, z), l = s->link_start[c];
                if (s->solid[c]) continue;
                for (int k = 1; k < NQ; ++k) {
                    int64_t cn = orc_neighbour(&s->b, x, y, z, k);
                    if (cn >= 0 && !s->solid[cn]) continue;
                    double q = orc_link_q_binned(&s->b, xyzr, &bins, x, y, z, k);
                    s->link_k[l] = (int8_t)k;
                    s->link_a[l] = orc_link_fallback(&s->b, s->solid, x, y, z, k, q, safeguards) ? 0.0
                                                                                  : (1.0 - 2.0 * q) / (1.0 + 2.0 * q);
                    ++l;
                }
            }
    orc_bins_free(&bins);
    orc_rates(tau, lambda, &s->omega_p, &s->omega_m, &s->nu);
    s->g[0] = gx;
    s->g[1] = gy;
    s->g[2] = gz;
    return s;
}

/* Incompressible equilibrium (Eq. (equilibrium)) with rho0 = 1, c_s^2 = 1/3,
 * written for full populations: f_k^eq = w_k [rho + 3 e.u + 9/2 (e.u)^2 - 3/2 u.u]. */
void orc_equilibrium(double rho, const double *u, double *feq)
{
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int k = 0; k < NQ; ++k) {
        double eu = ORC_EX[k] * u[0] + ORC_EY[k] * u[1] + ORC_EZ[k] * u[2];
        feq[k] = orc_weight(k) * (rho + 3.0 * eu + 4.5 * eu * eu - 1.5 * uu);
    }
}

/* Simple bounce-back (Eq. (noslip)) on every wall link: a = 0, i.e. the
 * wall half-way along each link whatever its q.  Call before stepping. */
void orc_lbm_set_simple_bounce_back(orc_lbm *s)
{
    const int64_t nl = s->link_start[s->ncell];
    for (int64_t l = 0; l < nl; ++l) s->link_a[l] = 0.0;
}

/* Initial state f_k = f_k^eq(rho = 1, u0); u0 is [3][ncell] or NULL (rest). */
void orc_lbm_init(orc_lbm *s, const double *u0)
{
    for (int64_t c = 0; c < s->ncell; ++c) {
        double u[3] = {0.0, 0.0, 0.0}, feq[NQ];
        if (s->solid[c]) {
            for (int k = 0; k < NQ; ++k) s->f[k * s->ncell + c] = 0.0;
            continue;
        }
        if (u0) {
            u[0] = u0[c];
            u[1] = u0[s->ncell + c];
            u[2] = u0[2 * s->ncell + c];
        }
        orc_equilibrium(1.0, u, feq);
        for (int k = 0; k < NQ; ++k) s->f[k * s->ncell + c] = feq[k];
    }
    s->has_prev = 0;
    s->steps = 0;
}

/* Collision (Eq. (collision)) with the TRT operator (Eqs. (TRT), (TRT2)):
 * f~_k = f_k - w+ (f_k^+ - f_k^{eq,+}) - w- (f_k^- - f_k^{eq,-}) + F_k,
 * F_k = 3 w_k e_k.g.  The equilibrium uses rho = sum f and j = sum e f of the
 * pre-collision state (Eq. (Macro), rho0 = 1). */
static void orc_collide(orc_lbm *s)
{
    const int64_t N = s->ncell;
#pragma omp parallel for schedule(static)
    for (int64_t c = 0; c < N; ++c) {
        if (s->solid[c]) continue;
        double f[NQ], feq[NQ], rho = 0.0, j[3] = {0.0, 0.0, 0.0};
        for (int k = 0; k < NQ; ++k) {
            f[k] = s->f[k * N + c];
            rho += f[k];
            j[0] += ORC_EX[k] * f[k];
            j[1] += ORC_EY[k] * f[k];
            j[2] += ORC_EZ[k] * f[k];
        }
        orc_equilibrium(rho, j, feq);
        for (int k = 0; k < NQ; ++k) {
            int kb = orc_opp(k);
            double fp = 0.5 * (f[k] + f[kb]), fm = 0.5 * (f[k] - f[kb]);
            double ep = 0.5 * (feq[k] + feq[kb]), em = 0.5 * (feq[k] - feq[kb]);
            double src = 3.0 * orc_weight(k) *
                         (ORC_EX[k] * s->g[0] + ORC_EY[k] * s->g[1] + ORC_EZ[k] * s->g[2]);
            s->fn[k * N + c] = f[k] - s->omega_p * (fp - ep) - s->omega_m * (fm - em) + src;
        }
    }
    /* the post-collision state becomes f (f~ at t_n); fn is reused for the
     * streamed state below */
    double *t = s->f;
    s->f = s->fn;
    s->fn = t;
}

/* Streaming (Eq. (streaming)) with central linear interpolation at walls
 * (Eq. (CLI)): for a fluid node x_f1 whose neighbour x_b = x_f1 + e_k is solid,
 *   f_kbar(x_f1, t+1) = a f~_k(x_f2) - a f~_kbar(x_f1) + f~_k(x_f1),
 *   a = (1-2q)/(1+2q),  x_f2 = x_f1 - e_k,
 * and a = 0 (simple bounce-back, Eq. (noslip)) on the fallback links of
 * orc_link_fallback. */
static void orc_stream(orc_lbm *s)
{
    const int64_t N = s->ncell;
    const orc_box *b = &s->b;
#pragma omp parallel for schedule(static)
    for (int z = 0; z < b->nz; ++z)
        for (int y = 0; y < b->ny; ++y)
            for (int x = 0; x < b->nx; ++x) {
                int64_t c = orc_cell(b, x, y, z);
                if (s->solid[c]) continue;
                s->fn[c] = s->f[c]; /* rest population stays */
                int64_t l = s->link_start[c];
                for (int k = 1; k < NQ; ++k) {
                    int64_t cn = orc_neighbour(b, x, y, z, k);
                    if (cn >= 0 && !s->solid[cn]) {
                        s->fn[k * N + cn] = s->f[k * N + c];
                        continue;
                    }
                    /* wall link (x, k); links of a cell are stored in k order */
                    int kb = orc_opp(k);
                    double a = s->link_a[l++];
                    double fk_x2 = 0.0;
                    if (a != 0.0) {
                        int64_t c2 = orc_neighbour(b, x, y, z, kb);
                        fk_x2 = s->f[k * N + c2];
                    }
                    s->fn[kb * N + c] = a * fk_x2 - a * s->f[kb * N + c] + s->f[k * N + c];
                }
            }
    double *t = s->f;
    s->f = s->fn;
    s->fn = t;
}

void orc_lbm_step(orc_lbm *s, int64_t n)
{
    for (int64_t t = 0; t < n; ++t) {
        orc_collide(s);
        orc_stream(s);
        ++s->steps;
    }
}

int64_t orc_lbm_steps(const orc_lbm *s) { return s->steps; }

/* Moments of the streamed state at t_n (Eq. (Macro)): rho = sum f and the
 * velocity u = j + g/2 (the mean of the pre- and post-collision momentum, the
 * velocity to which the source term of the collision is consistent).  Solid
 * cells give rho = 0, u = 0.  rho is [ncell], u is [3][ncell]; either may be
 * NULL. */
void orc_lbm_moments(const orc_lbm *s, double *rho, double *u)
{
    const int64_t N = s->ncell;
    for (int64_t c = 0; c < N; ++c) {
        double r = 0.0, j[3] = {0.0, 0.0, 0.0};
        if (!s->solid[c])
            for (int k = 0; k < NQ; ++k) {
                double fk = s->f[k * N + c];
                r += fk;
                j[0] += ORC_EX[k] * fk;
                j[1] += ORC_EY[k] * fk;
                j[2] += ORC_EZ[k] * fk;
            }
        if (rho) rho[c] = r;
        if (u) {
            int fl = !s->solid[c];
            u[c] = fl ? j[0] + 0.5 * s->g[0] : 0.0;
            u[N + c] = fl ? j[1] + 0.5 * s->g[1] : 0.0;
            u[2 * N + c] = fl ? j[2] + 0.5 * s->g[2] : 0.0;
        }
    }
}

/* Plane averages over z (Sec. 3.1, planar average of the stream-wise
 * velocity): out[3z+0] = sum_fluid u_x / (nx ny) (superficial),
 * out[3z+1] = sum_fluid u_x / n_fluid(z) (intrinsic; 0 for an all-solid plane),
 * out[3z+2] = n_fluid(z) / (nx ny) (plane porosity). */
void orc_lbm_plane_average(const orc_lbm *s, double *out)
{
    const orc_box *b = &s->b;
    const int64_t N = s->ncell;
    for (int z = 0; z < b->nz; ++z) {
        double sum = 0.0;
        int64_t nfl = 0;
        for (int y = 0; y < b->ny; ++y)
            for (int x = 0; x < b->nx; ++x) {
                int64_t c = orc_cell(b, x, y, z);
                if (s->solid[c]) continue;
                double jx = 0.0;
                for (int k = 0; k < NQ; ++k) jx += ORC_EX[k] * s->f[k * N + c];
                sum += jx + 0.5 * s->g[0];
                ++nfl;
            }
        double area = (double)b->nx * (double)b->ny;
        out[3 * z + 0] = sum / area;
        out[3 * z + 1] = nfl ? sum / (double)nfl : 0.0;
        out[3 * z + 2] = (double)nfl / area;
    }
}

/* Darcy permeability (Eq. (Darcy)) along x from the superficial mean velocity
 * of the planes z_lo..z_hi (both -1: the whole box): with mu = rho0 nu, no
 * mean pressure gradient and the body force F = g_x, K = nu <u_x> / g_x. */
double orc_lbm_permeability(const orc_lbm *s, int z_lo, int z_hi)
{
    const orc_box *b = &s->b;
    if (z_lo < 0 && z_hi < 0) { z_lo = 0; z_hi = b->nz - 1; }
    double *pa = (double *)malloc(sizeof(double) * 3 * (size_t)b->nz);
    if (!pa) return NAN;
    orc_lbm_plane_average(s, pa);
    double sum = 0.0;
    for (int z = z_lo; z <= z_hi; ++z) sum += pa[3 * z];
    free(pa);
    double mean = sum / (double)(z_hi - z_lo + 1);
    return s->nu * mean / s->g[0];
}

/* Convergence residual ||u^n - u^prev||_2 / ||u^n||_2 over fluid cells and all
 * three components, against the snapshot taken by the previous call (the
 * first call returns +inf); the current velocity becomes the new snapshot. */
double orc_lbm_residual(orc_lbm *s)
{
    const int64_t N = s->ncell;
    double *u = (double *)malloc(sizeof(double) * 3 * (size_t)N);
    if (!u) return NAN;
    orc_lbm_moments(s, NULL, u);
    double num = 0.0, den = 0.0;
    for (int64_t c = 0; c < N; ++c) {
        if (s->solid[c]) continue;
        for (int d = 0; d < 3; ++d) {
            double du = u[d * N + c] - s->uprev[d * N + c];
            num += du * du;
            den += u[d * N + c] * u[d * N + c];
        }
    }
    double res = s->has_prev ? sqrt(num) / sqrt(den) : INFINITY;
    memcpy(s->uprev, u, sizeof(double) * 3 * (size_t)N);
    s->has_prev = 1;
    free(u);
    return res;
}

void orc_lbm_get_f(const orc_lbm *s, double *f) { memcpy(f, s->f, sizeof(double) * NQ * (size_t)s->ncell); }
void orc_lbm_set_f(orc_lbm *s, const double *f) { memcpy(s->f, f, sizeof(double) * NQ * (size_t)s->ncell); }
void orc_lbm_solid(const orc_lbm *s, uint8_t *solid) { memcpy(solid, s->solid, (size_t)s->ncell); }
double orc_lbm_nu(const orc_lbm *s) { return s->nu; }
double orc_lbm_omega_minus(const orc_lbm *s) { return s->omega_m; }

int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void orc_set_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}
