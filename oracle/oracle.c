/*
 * oracle.c -- plain, slow, FP64 CPU oracle of the tree-code force evaluation
 * (N. Nakasato, "Implementation of a Parallel Tree Method on a GPU").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library.
 *
 * Every function below is written from the paper's definitions (cited per
 * function) in the most direct form: no blocking, no fusion, no reordering.
 * Floating point is FP64 except where a floating-point result decides an
 * integer (root box, Morton keys): there the decision is taken in FP32 with
 * IEEE round-to-nearest and no contraction, exactly as the GPU kernel does
 * (this file must be compiled with -ffp-contract=off).
 *
 * Conventions (readings of the paper where it is silent or ambiguous):
 *   - sign: accelerations are attractive and the potential is negative,
 *     phi_i = -sum m_j / sqrt(r^2 + eps^2)  (the paper's p_i is -phi_i);
 *   - the self term is excluded by index (Eq. 1, j != i);
 *   - particle-cell terms are softened with the same eps as particle-particle
 *     terms unless `unsoftened_pc` is set (the Appendix A kernel's form);
 *   - a node holding the target (or, in the group walk, any group member) is
 *     never accepted, it is opened;
 *   - tree: node = non-empty cell of the 2^l grid (l = 0..10) whose parent cell
 *     holds more than n_leaf particles; a node is a leaf when it holds at most
 *     n_leaf particles or l == 10; nodes are stored breadth first, i.e. sorted
 *     by (level, first particle), so the children of a node are contiguous.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_CURVE_MORTON 0
#define OR_CURVE_HILBERT 1

int or_version(void) { return 3; }

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void or_set_threads(int t)
{
#ifdef _OPENMP
    if (t > 0) omp_set_num_threads(t);
#else
    (void)t;
#endif
}

/* ------------------------------------------------------------------------
 * Eq. (1), Sec. 3: softened direct summation over all j != i.
 * src: n_src x (x,y,z,m) FP32;  tgt: n_tgt x (x,y,z,*) FP32;
 * self: optional index into src excluded for each target (-1 = none);
 * out:  n_tgt x (ax,ay,az,phi) FP64.
 * ---------------------------------------------------------------------- */
void or_direct(int64_t n_src, const float* src, int64_t n_tgt, const float* tgt,
               const int64_t* self, double eps, double* out)
{
    const double e2 = eps * eps;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 8)
    for (i = 0; i < n_tgt; i++) {
        const double xi = tgt[4 * i], yi = tgt[4 * i + 1], zi = tgt[4 * i + 2];
        const int64_t skip = self ? self[i] : -1;
        double ax = 0, ay = 0, az = 0, phi = 0;
        for (int64_t j = 0; j < n_src; j++) {
            if (j == skip) continue;
            const double dx = (double)src[4 * j] - xi;
            const double dy = (double)src[4 * j + 1] - yi;
            const double dz = (double)src[4 * j + 2] - zi;
            const double m = src[4 * j + 3];
            const double r2 = dx * dx + dy * dy + dz * dz + e2;
            const double rinv = 1.0 / sqrt(r2);
            const double mr3 = m * rinv * rinv * rinv;
            ax += mr3 * dx;
            ay += mr3 * dy;
            az += mr3 * dz;
            phi -= m * rinv;
        }
        out[4 * i] = ax;
        out[4 * i + 1] = ay;
        out[4 * i + 2] = az;
        out[4 * i + 3] = phi;
    }
}

/* ------------------------------------------------------------------------
 * Individual softening with the symmetrized Plummer potential (Sec. 7 names
 * it as an application of the method, after Saitoh & Makino 2010): particle
 * i has its own softening length eps_i, and a pair softens with
 *   eps_ij^2 = (eps_i^2 + eps_j^2) / 2,
 * so phi_i = -sum_j m_j / sqrt(r^2 + eps_ij^2) and the pair force is the same
 * for both bodies (total momentum is conserved).  eps_src, eps_tgt: FP32
 * lengths per source and per target; otherwise as or_direct.
 * ---------------------------------------------------------------------- */
void or_direct_sym(int64_t n_src, const float* src, const float* eps_src, int64_t n_tgt, const float* tgt,
                   const float* eps_tgt, const int64_t* self, double* out)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 8)
    for (i = 0; i < n_tgt; i++) {
        const double xi = tgt[4 * i], yi = tgt[4 * i + 1], zi = tgt[4 * i + 2];
        const double ei = eps_tgt[i];
        const int64_t own = self ? self[i] : -1;
        double a[4] = {0, 0, 0, 0};
        for (int64_t j = 0; j < n_src; j++) {
            if (j == own) continue;
            const double ej = eps_src[j];
            const double dx = (double)src[4 * j] - xi;
            const double dy = (double)src[4 * j + 1] - yi;
            const double dz = (double)src[4 * j + 2] - zi;
            const double mj = src[4 * j + 3];
            const double r2 = dx * dx + dy * dy + dz * dz + 0.5 * (ei * ei + ej * ej);
            const double g1 = 1.0 / sqrt(r2);
            const double k = mj * g1 * g1 * g1;
            a[0] += k * dx;
            a[1] += k * dy;
            a[2] += k * dz;
            a[3] -= mj * g1;
        }
        for (int c = 0; c < 4; c++) out[4 * i + c] = a[c];
    }
}

/* A node's softening under the symmetrized potential: the mass-weighted mean
 * of its particles' eps_j^2 (0 for a massless node, whose terms vanish).  With
 * this mean the term of first order in the spread of eps_j^2 inside the cell
 * cancels, as the dipole does about the centre of mass.  eps_s: per sorted
 * particle; e2bar: per node (FP64 direct sums). */
void or_cell_softening(int64_t nn, const float* spos, const float* eps_s, const int32_t* first,
                       const int32_t* count, double* e2bar)
{
    int64_t v;
#pragma omp parallel for schedule(dynamic, 64)
    for (v = 0; v < nn; v++) {
        double sm = 0.0, se = 0.0;
        for (int64_t j = first[v]; j < (int64_t)first[v] + count[v]; j++) {
            const double m = spos[4 * j + 3], e = eps_s[j];
            sm += m;
            se += m * e * e;
        }
        e2bar[v] = sm != 0.0 ? se / sm : 0.0;
    }
}

/* ------------------------------------------------------------------------
 * Sec. 4.1: the root cell is a cube enclosing all particles.  Origin = the
 * per-axis minimum, side L = the largest per-axis extent (FP32, exact min/max,
 * one rounded subtraction).  A degenerate side (0, or one whose 1024/L is not
 * finite) is replaced by 1.  box = (xmin, ymin, zmin, L).
 * ---------------------------------------------------------------------- */
void or_bbox(int64_t n, const float* pos, float* box)
{
    float lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    for (int64_t i = 0; i < n; i++)
        for (int a = 0; a < 3; a++) {
            const float v = pos[4 * i + a];
            if (i == 0 || v < lo[a]) lo[a] = v;
            if (i == 0 || v > hi[a]) hi[a] = v;
        }
    float L = 0.0f;
    for (int a = 0; a < 3; a++) {
        const float d = hi[a] - lo[a];
        if (d > L) L = d;
    }
    const float inv = 1024.0f / L;
    if (!(L > 0.0f) || !isfinite(inv)) L = 1.0f;
    box[0] = lo[0];
    box[1] = lo[1];
    box[2] = lo[2];
    box[3] = L;
}

/* Spread the low `nbits` bits of v so that bit k moves to bit 3k. */
static uint64_t or_spread3(uint32_t v, int nbits)
{
    uint64_t r = 0;
    for (int k = 0; k < nbits; k++) r |= (uint64_t)((v >> k) & 1u) << (3 * k);
    return r;
}

/* Inverse of or_spread3 restricted to `nbits` triples. */
static uint32_t or_compact3(uint64_t v, int nbits)
{
    uint32_t r = 0;
    for (int k = 0; k < nbits; k++) r |= (uint32_t)((v >> (3 * k)) & 1u) << k;
    return r;
}

/* ------------------------------------------------------------------------
 * Peano-Hilbert order (the ordering Sec. 5 names as better than Morton's),
 * after J. Skilling, "Programming the Hilbert curve", AIP Conf. Proc. 707
 * (2004): the cell's coordinates (nbits bits each) are turned into the
 * "transposed" index by undoing, from the top level down, the reflections
 * and axis exchanges of the curve's sub-cubes, and are then Gray-coded; the
 * index interleaves the three transposed words as the Morton key does (first
 * word in the high bit of each triple).  Level by level, each octree cell is
 * one contiguous index range, so the tree is read off the sorted keys exactly
 * as with Morton keys, only the children's order differs.
 * ---------------------------------------------------------------------- */
static uint64_t or_hilbert3(uint32_t x, uint32_t y, uint32_t z, int nbits)
{
    uint32_t w[3] = {x, y, z};
    for (uint32_t q = 1u << (nbits - 1); q > 1u; q >>= 1) {
        const uint32_t low = q - 1u;
        for (int a = 0; a < 3; a++) {
            if (w[a] & q) {
                w[0] ^= low;                              /* reflect */
            } else {
                const uint32_t d = (w[0] ^ w[a]) & low;   /* exchange axes 0 and a */
                w[0] ^= d;
                w[a] ^= d;
            }
        }
    }
    w[1] ^= w[0];
    w[2] ^= w[1];
    uint32_t g = 0;
    for (uint32_t q = 1u << (nbits - 1); q > 1u; q >>= 1)
        if (w[2] & q) g ^= q - 1u;
    for (int a = 0; a < 3; a++) w[a] ^= g;
    return (or_spread3(w[0], nbits) << 2) | (or_spread3(w[1], nbits) << 1) | or_spread3(w[2], nbits);
}

/* Inverse of or_hilbert3: cell coordinates of an index. */
static void or_hilbert3_inv(uint64_t h, int nbits, uint32_t* c)
{
    uint32_t w[3] = {or_compact3(h >> 2, nbits), or_compact3(h >> 1, nbits), or_compact3(h, nbits)};
    const uint32_t g = w[2] >> 1;                          /* Gray decode */
    w[2] ^= w[1];
    w[1] ^= w[0];
    w[0] ^= g;
    for (uint32_t q = 2u; q != (1u << nbits); q <<= 1) {
        const uint32_t low = q - 1u;
        for (int a = 2; a >= 0; a--) {
            if (w[a] & q) {
                w[0] ^= low;
            } else {
                const uint32_t d = (w[0] ^ w[a]) & low;
                w[0] ^= d;
                w[a] ^= d;
            }
        }
    }
    c[0] = w[0];
    c[1] = w[1];
    c[2] = w[2];
}

/* Integer cell (nbits bits per axis) of a key of either order. */
static void or_key_cell(uint64_t key, int curve, int nbits, uint32_t* c)
{
    if (curve == OR_CURVE_HILBERT) {
        or_hilbert3_inv(key, nbits, c);
    } else {
        c[0] = or_compact3(key >> 2, nbits);
        c[1] = or_compact3(key >> 1, nbits);
        c[2] = or_compact3(key, nbits);
    }
}

/* Exported for the pins: key of a cell, and cell of a key. */
uint64_t or_key_of_cell(uint32_t x, uint32_t y, uint32_t z, int curve, int nbits)
{
    return curve == OR_CURVE_HILBERT
               ? or_hilbert3(x, y, z, nbits)
               : (or_spread3(x, nbits) << 2) | (or_spread3(y, nbits) << 1) | or_spread3(z, nbits);
}
void or_cell_of_key(uint64_t key, int curve, int nbits, uint32_t* c) { or_key_cell(key, curve, nbits, c); }

/* ------------------------------------------------------------------------
 * Sec. 5 (Morton ordering): key of max_level bits per axis (10: 30-bit keys;
 * 21: 63-bit keys).  q = (x - xmin) * inv in FP32 (two rounded ops) with
 * inv = (1024/L) * 2^(max_level - 10) (the power of two is exact), integer
 * cell c = min(trunc(q), 2^max_level - 1); bit k of cx, cy, cz goes to key
 * bit 3k+2, 3k+1, 3k.  curve = OR_CURVE_HILBERT gives the Peano-Hilbert
 * index of the same cell.  The top 3*10 bits of a 63-bit key are the 30-bit
 * key of the same particle (the 10-bit cell is the 21-bit cell >> 11).
 * ---------------------------------------------------------------------- */
void or_keys(int64_t n, const float* pos, const float* box, uint64_t* keys, int curve, int max_level)
{
    const float inv = (1024.0f / box[3]) * (float)(1u << (max_level - 10));
    const uint32_t cmax = (1u << max_level) - 1u;
    for (int64_t i = 0; i < n; i++) {
        uint32_t c[3];
        for (int a = 0; a < 3; a++) {
            const float t = pos[4 * i + a] - box[a];
            const float q = t * inv;
            uint32_t ci = (uint32_t)q;
            if (ci > cmax) ci = cmax;
            c[a] = ci;
        }
        keys[i] = or_key_of_cell(c[0], c[1], c[2], curve, max_level);
    }
}

/* ------------------------------------------------------------------------
 * Stable sort of indices 0..n-1 by key (plain top-down merge sort).
 * perm[k] = original index of the k-th particle in Morton order.
 * ---------------------------------------------------------------------- */
static void or_merge_sort(uint32_t* a, uint32_t* tmp, int64_t lo, int64_t hi, const uint64_t* keys)
{
    if (hi - lo < 2) return;
    const int64_t mid = lo + (hi - lo) / 2;
    or_merge_sort(a, tmp, lo, mid, keys);
    or_merge_sort(a, tmp, mid, hi, keys);
    int64_t i = lo, j = mid, k = lo;
    while (i < mid && j < hi) {
        if (keys[a[j]] < keys[a[i]]) tmp[k++] = a[j++];
        else tmp[k++] = a[i++];
    }
    while (i < mid) tmp[k++] = a[i++];
    while (j < hi) tmp[k++] = a[j++];
    memcpy(a + lo, tmp + lo, (size_t)(hi - lo) * sizeof(uint32_t));
}

int or_sort(int64_t n, const uint64_t* keys, uint32_t* perm)
{
    uint32_t* tmp = (uint32_t*)malloc((size_t)(n > 0 ? n : 1) * sizeof(uint32_t));
    if (!tmp) return -1;
    for (int64_t i = 0; i < n; i++) perm[i] = (uint32_t)i;
    or_merge_sort(perm, tmp, 0, n, keys);
    free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------
 * Sec. 4.1 tree construction: recursively split a cube into 8 equal
 * sub-cells.  Here the recursion stops at a cell holding <= n_leaf particles
 * or at max_level (the key's resolution: 10 or 21).  Nodes are emitted level
 * by level, children in octant order, so node order = (level, first).
 * Returns the node count, or -1 if `cap` is too small.
 * ---------------------------------------------------------------------- */
int64_t or_tree_build(int64_t n, const uint64_t* skeys, int n_leaf, int max_level, int64_t cap,
                      int32_t* level, int32_t* first, int32_t* count,
                      int32_t* child_first, int32_t* nchild)
{
    if (n <= 0) return 0;
    if (cap < 1) return -1;
    int64_t nn = 1;
    level[0] = 0;
    first[0] = 0;
    count[0] = (int32_t)n;
    int64_t lev_begin = 0, lev_end = 1;
    for (int l = 0; l <= max_level; l++) {
        for (int64_t v = lev_begin; v < lev_end; v++) {
            if (count[v] <= n_leaf || l == max_level) {
                child_first[v] = -1;
                nchild[v] = 0;
                continue;
            }
            /* digit of the sub-cell at level l+1 */
            const int shift = 3 * (max_level - 1 - l);
            child_first[v] = (int32_t)nn;
            nchild[v] = 0;
            int64_t k = first[v];
            const int64_t end = (int64_t)first[v] + count[v];
            while (k < end) {
                const uint64_t d = (skeys[k] >> shift) & 7u;
                int64_t e = k;
                while (e < end && ((skeys[e] >> shift) & 7u) == d) e++;
                if (nn >= cap) return -1;
                level[nn] = l + 1;
                first[nn] = (int32_t)k;
                count[nn] = (int32_t)(e - k);
                nn++;
                nchild[v]++;
                k = e;
            }
        }
        lev_begin = lev_end;
        lev_end = nn;
        if (lev_begin == lev_end) break;
    }
    return nn;
}

/* ------------------------------------------------------------------------
 * Sec. 4.4 cell data: total mass, centre of mass, and Eq. (2)'s effective
 * size S_eff = (l/theta + s)^2, where l is the side of the node's cube and s
 * the distance from the cube's centre to the centre of mass.  For order 2
 * also the raw second moment about the centre of mass,
 * I_ab = sum m (x_a - c_a)(x_b - c_b), stored (xx, yy, zz, xy, xz, yz).
 * Every node is summed directly over its own particles (not from its
 * children).  A massless node takes its geometric centre as centre of mass.
 * spos: particles in Morton order (x,y,z,m) FP32; skeys: their keys
 * (max_level bits per axis).
 * Outputs per node: com_m (cx,cy,cz,M), quad[6] (may be NULL), s_eff, side.
 * ---------------------------------------------------------------------- */
void or_moments(int64_t nn, const float* spos, const uint64_t* skeys,
                const int32_t* level, const int32_t* first, const int32_t* count,
                const float* box, double theta, double* com_m, double* quad,
                double* s_eff, double* side, int curve, int max_level)
{
    int64_t v;
#pragma omp parallel for schedule(dynamic, 64)
    for (v = 0; v < nn; v++) {
        const int l = level[v];
        const int64_t b = first[v], e = (int64_t)first[v] + count[v];
        double M = 0, sx = 0, sy = 0, sz = 0;
        for (int64_t k = b; k < e; k++) {
            const double m = spos[4 * k + 3];
            M += m;
            sx += m * spos[4 * k];
            sy += m * spos[4 * k + 1];
            sz += m * spos[4 * k + 2];
        }
        /* geometric centre of the level-l cell containing the node */
        const double lside = (double)box[3] / (double)(1u << l);
        uint32_t cell[3];
        or_key_cell(skeys[b], curve, max_level, cell);  /* the first particle's cell, then its level-l ancestor */
        const double px = cell[0] >> (max_level - l), py = cell[1] >> (max_level - l),
                     pz = cell[2] >> (max_level - l);
        const double gx = (double)box[0] + (px + 0.5) * lside;
        const double gy = (double)box[1] + (py + 0.5) * lside;
        const double gz = (double)box[2] + (pz + 0.5) * lside;
        double cx, cy, cz;
        if (M > 0) {
            cx = sx / M;
            cy = sy / M;
            cz = sz / M;
        } else {
            cx = gx;
            cy = gy;
            cz = gz;
        }
        com_m[4 * v] = cx;
        com_m[4 * v + 1] = cy;
        com_m[4 * v + 2] = cz;
        com_m[4 * v + 3] = M;
        if (quad) {
            double q[6] = {0, 0, 0, 0, 0, 0};
            for (int64_t k = b; k < e; k++) {
                const double m = spos[4 * k + 3];
                const double y0 = spos[4 * k] - cx, y1 = spos[4 * k + 1] - cy, y2 = spos[4 * k + 2] - cz;
                q[0] += m * y0 * y0;
                q[1] += m * y1 * y1;
                q[2] += m * y2 * y2;
                q[3] += m * y0 * y1;
                q[4] += m * y0 * y2;
                q[5] += m * y1 * y2;
            }
            for (int c = 0; c < 6; c++) quad[6 * v + c] = q[c];
        }
        const double s = sqrt((gx - cx) * (gx - cx) + (gy - cy) * (gy - cy) + (gz - cz) * (gz - cz));
        const double t = lside / theta + s;
        s_eff[v] = t * t;
        if (side) side[v] = lside;
    }
}

/* ------------------------------------------------------------------------
 * Particle groups for the group walk (an extension in the spirit of the
 * GRAPE interaction lists of Sec. 4.2: one list shared by nearby targets).
 * Groups partition the Morton-ordered particles:
 *   - if the root holds <= G particles it is the only group;
 *   - for every internal node P holding > G particles, its children are
 *     visited in octant order; children holding <= G particles are packed
 *     greedily, in order, into runs of total <= G (a child holding > G
 *     particles ends the current run); a leaf holding > G particles
 *     (possible only at level 10, or when n_leaf > G) is cut into chunks of G.
 * Groups are returned sorted by first particle.  Returns the group count or
 * -1 if `cap` is too small.
 * ---------------------------------------------------------------------- */
static int or_cmp_i64(const void* a, const void* b)
{
    const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

int64_t or_groups(int64_t nn, const int32_t* first, const int32_t* count,
                  const int32_t* child_first, const int32_t* nchild, int G, int64_t cap,
                  int32_t* g_first, int32_t* g_count)
{
    if (nn <= 0) return 0;
    /* (first << 32 | count) pairs, sorted at the end */
    int64_t* tmp = (int64_t*)malloc((size_t)(cap > 0 ? cap : 1) * sizeof(int64_t));
    if (!tmp) return -1;
    int64_t ng = 0;
#define OR_EMIT(F, C)                                                  \
    do {                                                               \
        if (ng >= cap) { free(tmp); return -1; }                       \
        tmp[ng++] = ((int64_t)(F) << 32) | (int64_t)(uint32_t)(C);     \
    } while (0)
    if (count[0] <= G) {
        OR_EMIT(first[0], count[0]);
    } else if (nchild[0] == 0) {
        for (int64_t k = 0; k < count[0]; k += G)
            OR_EMIT(first[0] + k, (count[0] - k < G) ? (count[0] - k) : G);
    } else {
        for (int64_t p = 0; p < nn; p++) {
            if (nchild[p] == 0 || count[p] <= G) continue;
            int64_t run_first = -1, run_count = 0;
            for (int c = 0; c < nchild[p]; c++) {
                const int64_t ch = child_first[p] + c;
                if (count[ch] <= G) {
                    if (run_first >= 0 && run_count + count[ch] <= G) {
                        run_count += count[ch];
                    } else {
                        if (run_first >= 0) OR_EMIT(run_first, run_count);
                        run_first = first[ch];
                        run_count = count[ch];
                    }
                } else {
                    if (run_first >= 0) OR_EMIT(run_first, run_count);
                    run_first = -1;
                    run_count = 0;
                    if (nchild[ch] == 0)
                        for (int64_t k = 0; k < count[ch]; k += G)
                            OR_EMIT(first[ch] + k, (count[ch] - k < G) ? (count[ch] - k) : G);
                }
            }
            if (run_first >= 0) OR_EMIT(run_first, run_count);
        }
    }
#undef OR_EMIT
    qsort(tmp, (size_t)ng, sizeof(int64_t), or_cmp_i64);
    for (int64_t g = 0; g < ng; g++) {
        g_first[g] = (int32_t)(tmp[g] >> 32);
        g_count[g] = (int32_t)(tmp[g] & 0xffffffff);
    }
    free(tmp);
    return ng;
}

/* ------------------------------------------------------------------------
 * Interaction kernels (Eq. 1 and its multipole generalisation).
 * r = x_i - c,  h^2 = |r|^2 + eps^2,  g_n = h^-n.
 * Monopole: phi = -M g1,  a = -M g3 r.
 * Quadrupole (second-order Taylor term of the softened kernel about the
 * centre of mass, where the dipole vanishes):
 *   phi += -(3 q g5 - T g3)/2,   a += 3 g5 (I r) + (1.5 T g5 - 7.5 q g7) r,
 * with T = tr I and q = r.I.r.  At eps = 0 this is the traceless form
 * -r.Q.r / (2 |r|^5) with Q = 3I - T 1.
 * ---------------------------------------------------------------------- */
static void or_pc(double xi, double yi, double zi, const double* cm, const double* qd,
                  double e2, double* acc)
{
    const double rx = xi - cm[0], ry = yi - cm[1], rz = zi - cm[2], M = cm[3];
    const double h2 = rx * rx + ry * ry + rz * rz + e2;
    const double g1 = 1.0 / sqrt(h2);
    const double g2 = g1 * g1;
    const double g3 = g1 * g2;
    acc[0] -= M * g3 * rx;
    acc[1] -= M * g3 * ry;
    acc[2] -= M * g3 * rz;
    acc[3] -= M * g1;
    acc[4] += fabs(M) * g3 * sqrt(rx * rx + ry * ry + rz * rz);
    if (qd) {
        const double g5 = g3 * g2, g7 = g5 * g2;
        const double Ir0 = qd[0] * rx + qd[3] * ry + qd[4] * rz;
        const double Ir1 = qd[3] * rx + qd[1] * ry + qd[5] * rz;
        const double Ir2 = qd[4] * rx + qd[5] * ry + qd[2] * rz;
        const double T = qd[0] + qd[1] + qd[2];
        const double q = rx * Ir0 + ry * Ir1 + rz * Ir2;
        const double c = 1.5 * T * g5 - 7.5 * q * g7;
        acc[0] += 3.0 * g5 * Ir0 + c * rx;
        acc[1] += 3.0 * g5 * Ir1 + c * ry;
        acc[2] += 3.0 * g5 * Ir2 + c * rz;
        acc[3] -= 0.5 * (3.0 * q * g5 - T * g3);
    }
}

/* A cell term of the walks.  The paper's kernel (Appendix A) reads each
 * cell as a float4 (x, y, z, m) like a particle, so the term is applied with
 * the centre of mass and mass rounded to FP32 (the moments themselves are
 * exact FP64 sums).  Near the FP32 resolution of the coordinates (cells of
 * 63-bit key trees seen from inside the same dense knot) this rounding is
 * the leading difference between the FP64 and the stored cell. */
static int or_cell_fp32 = 1;

/* Switch the FP32 rounding of the cell record on (1, the default) or off (0:
 * cell terms use the exact FP64 centre of mass and mass).  For tests that
 * show where the rounding matters and where it does not. */
void or_set_cell_rounding(int on) { or_cell_fp32 = on != 0; }

static void or_pc_cell(double xi, double yi, double zi, const double* cm, const double* qd, double e2,
                       double* acc)
{
    if (!or_cell_fp32) {
        or_pc(xi, yi, zi, cm, qd, e2, acc);
        return;
    }
    const double c[4] = {(double)(float)cm[0], (double)(float)cm[1], (double)(float)cm[2], (double)(float)cm[3]};
    or_pc(xi, yi, zi, c, qd, e2, acc);
}

static void or_pp(double xi, double yi, double zi, const float* pj, double e2, double* acc)
{
    const double dx = (double)pj[0] - xi, dy = (double)pj[1] - yi, dz = (double)pj[2] - zi;
    const double m = pj[3];
    const double r2 = dx * dx + dy * dy + dz * dz + e2;
    const double rinv = 1.0 / sqrt(r2);
    const double mr3 = m * rinv * rinv * rinv;
    acc[0] += mr3 * dx;
    acc[1] += mr3 * dy;
    acc[2] += mr3 * dz;
    acc[3] -= m * rinv;
    acc[4] += fabs(mr3) * sqrt(dx * dx + dy * dy + dz * dz);
}

/* ------------------------------------------------------------------------
 * Group walk (group form of Fig. 3's tree walk, with Eq. 2's criterion
 * applied conservatively to the whole group): a node is accepted for the
 * group when the squared distance from its centre of mass to the group's
 * axis-aligned bounding box exceeds S_eff (strict, as the Appendix A kernel's
 * `s < r2`) and the node holds no member of the group (for theta above
 * 1/sqrt(3) Eq. 2 alone could accept a cell holding the target itself); an
 * accepted node gives a particle-cell term to every member; a
 * rejected leaf gives particle-particle terms with all its particles (the
 * target itself excluded by index); a rejected internal node is opened.
 *
 * spos: Morton-ordered particles; perm: Morton position -> caller index.
 * out (caller order, n x 4): ax, ay, az, phi.
 * margin (caller order, optional): min over the group's decisions of
 *   |d^2 - S_eff| / S_eff, so near-tie decisions can be recognised.
 * n_pp, n_pc (caller order, optional): interactions evaluated per target.
 * a_abs (caller order, optional): sum over all terms of |a_term|, the scale
 *   of the rounding error of any finite-precision evaluation of the sum.
 * group_mask (optional, per group): walk only groups whose mask is non-zero;
 *   the other targets are left untouched.
 * ---------------------------------------------------------------------- */
int or_force_groups(int64_t n, const float* spos, const uint32_t* perm, int64_t nn,
                    const int32_t* first, const int32_t* count, const int32_t* child_first,
                    const int32_t* nchild, const double* com_m, const double* quad,
                    const double* s_eff, int64_t ng, const int32_t* g_first, const int32_t* g_count,
                    const uint8_t* group_mask, double eps, double* out, double* margin,
                    int64_t* n_pp, int64_t* n_pc, double* a_abs)
{
    const double e2 = eps * eps;
    int err = 0;
    (void)n;
    int64_t g;
#pragma omp parallel for schedule(dynamic, 4)
    for (g = 0; g < ng; g++) {
        if (group_mask && !group_mask[g]) continue;
        const int64_t gb = g_first[g], ge = (int64_t)g_first[g] + g_count[g];
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) lo[a] = hi[a] = spos[4 * gb + a];
        for (int64_t k = gb; k < ge; k++)
            for (int a = 0; a < 3; a++) {
                const double v = spos[4 * k + a];
                if (v < lo[a]) lo[a] = v;
                if (v > hi[a]) hi[a] = v;
            }
        int32_t* stack = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
        int32_t* pc = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
        int32_t* pp = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
        if (!stack || !pc || !pp) {
            free(stack); free(pc); free(pp);
#pragma omp atomic write
            err = -1;
            continue;
        }
        int64_t sp = 0, npc = 0, npp = 0;
        double mmin = INFINITY;
        stack[sp++] = 0;
        while (sp > 0) {
            const int32_t v = stack[--sp];
            const double* c = com_m + 4 * v;
            double d2 = 0;
            for (int a = 0; a < 3; a++) {
                double t = 0;
                if (c[a] < lo[a]) t = lo[a] - c[a];
                else if (c[a] > hi[a]) t = c[a] - hi[a];
                d2 += t * t;
            }
            const double S = s_eff[v];
            const int holds_member = first[v] < ge && (int64_t)first[v] + count[v] > gb;
            if (!holds_member) {
                const double mg = fabs(d2 - S) / S;
                if (mg < mmin) mmin = mg;
            }
            if (d2 > S && !holds_member) pc[npc++] = v;
            else if (nchild[v] == 0) pp[npp++] = v;
            else
                for (int ch = nchild[v] - 1; ch >= 0; ch--) stack[sp++] = child_first[v] + ch;
        }
        for (int64_t i = gb; i < ge; i++) {
            const double xi = spos[4 * i], yi = spos[4 * i + 1], zi = spos[4 * i + 2];
            double acc[5] = {0, 0, 0, 0, 0};
            int64_t cnt_pp = 0;
            for (int64_t t = 0; t < npc; t++)
                or_pc_cell(xi, yi, zi, com_m + 4 * pc[t], quad ? quad + 6 * pc[t] : NULL, e2, acc);
            for (int64_t t = 0; t < npp; t++) {
                const int64_t b = first[pp[t]], e = b + count[pp[t]];
                for (int64_t j = b; j < e; j++) {
                    if (j == i) continue;
                    or_pp(xi, yi, zi, spos + 4 * j, e2, acc);
                    cnt_pp++;
                }
            }
            const int64_t o = perm[i];
            for (int a = 0; a < 4; a++) out[4 * o + a] = acc[a];
            if (margin) margin[o] = mmin;
            if (a_abs) a_abs[o] = acc[4];
            if (n_pp) n_pp[o] = cnt_pp;
            if (n_pc) n_pc[o] = npc;
        }
        free(stack);
        free(pc);
        free(pp);
    }
    return err;
}

/* Accepted-node and opened-leaf lists of one group (for invariant tests). */
int64_t or_group_lists(int64_t nn, const float* spos, const int32_t* first, const int32_t* count,
                       const int32_t* child_first, const int32_t* nchild, const double* com_m,
                       const double* s_eff, int32_t gb, int32_t gc, int32_t* pc, int64_t* npc_out,
                       int32_t* pp, int64_t* npp_out)
{
    double lo[3], hi[3];
    for (int a = 0; a < 3; a++) lo[a] = hi[a] = spos[4 * (int64_t)gb + a];
    for (int64_t k = gb; k < (int64_t)gb + gc; k++)
        for (int a = 0; a < 3; a++) {
            const double v = spos[4 * k + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    int32_t* stack = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
    if (!stack) return -1;
    int64_t sp = 0, npc = 0, npp = 0;
    stack[sp++] = 0;
    while (sp > 0) {
        const int32_t v = stack[--sp];
        const double* c = com_m + 4 * v;
        double d2 = 0;
        for (int a = 0; a < 3; a++) {
            double t = 0;
            if (c[a] < lo[a]) t = lo[a] - c[a];
            else if (c[a] > hi[a]) t = c[a] - hi[a];
            d2 += t * t;
        }
        const int holds_member = first[v] < gb + gc && first[v] + count[v] > gb;
        if (d2 > s_eff[v] && !holds_member) pc[npc++] = v;
        else if (nchild[v] == 0) pp[npp++] = v;
        else
            for (int ch = nchild[v] - 1; ch >= 0; ch--) stack[sp++] = child_first[v] + ch;
    }
    free(stack);
    *npc_out = npc;
    *npp_out = npp;
    return 0;
}

/* ------------------------------------------------------------------------
 * Per-particle walk of Fig. 3 / Fig. 5 (the paper's own form): for target i,
 * a node holding a single particle is a particle-particle term; otherwise
 * the node is accepted when d^2 > S_eff with d = |x_i - COM| (Eq. 2) and
 * it does not hold particle i itself; a
 * rejected leaf gives particle-particle terms with its members; a rejected
 * internal node is opened.  The self term is skipped by index.  With
 * unsoftened_pc the particle-cell term uses eps = 0 (the Appendix A kernel).
 * With eps_s (per sorted particle) and e2bar (per node, or_cell_softening)
 * the softening is individual and symmetrized: a particle term uses
 * (eps_i^2 + eps_j^2)/2 and a cell term (eps_i^2 + e2bar)/2 (eps is unused).
 * Targets are the Morton positions [t0, t1); out etc. are in caller order.
 * margin (optional): min over the target's criterion decisions (nodes not
 *   holding it) of |d^2 - S_eff| / S_eff; a_abs (optional): sum of |a_term|.
 * ---------------------------------------------------------------------- */
int or_force_particles(int64_t n, const float* spos, const uint32_t* perm, int64_t nn,
                       const int32_t* first, const int32_t* count, const int32_t* child_first,
                       const int32_t* nchild, const double* com_m, const double* quad,
                       const double* s_eff, int64_t t0, int64_t t1, double eps, int unsoftened_pc,
                       const float* eps_s, const double* e2bar,
                       double* out, int64_t* n_pp, int64_t* n_pc, double* margin, double* a_abs)
{
    const double e2 = eps * eps;
    const double e2c = unsoftened_pc ? 0.0 : e2;
    int err = 0;
    (void)n;
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = t0; i < t1; i++) {
        int32_t* stack = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
        if (!stack) {
#pragma omp atomic write
            err = -1;
            continue;
        }
        const double xi = spos[4 * i], yi = spos[4 * i + 1], zi = spos[4 * i + 2];
        const double ei2 = eps_s ? (double)eps_s[i] * (double)eps_s[i] : 0.0;
        double acc[5] = {0, 0, 0, 0, 0};
        double mmin = INFINITY;
        int64_t cpp = 0, cpc = 0, sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const int32_t v = stack[--sp];
            if (count[v] == 1) {
                if (first[v] != i) {
                    const double ej = eps_s ? eps_s[first[v]] : 0.0;
                    or_pp(xi, yi, zi, spos + 4 * (int64_t)first[v], eps_s ? 0.5 * (ei2 + ej * ej) : e2, acc);
                    cpp++;
                }
                continue;
            }
            const double* c = com_m + 4 * v;
            const double dx = c[0] - xi, dy = c[1] - yi, dz = c[2] - zi;
            const double d2 = dx * dx + dy * dy + dz * dz;
            const int holds_i = first[v] <= i && i < (int64_t)first[v] + count[v];
            if (!holds_i && s_eff[v] > 0.0) {
                const double mg = fabs(d2 - s_eff[v]) / s_eff[v];
                if (mg < mmin) mmin = mg;
            }
            if (d2 > s_eff[v] && !holds_i) {
                const double ec = eps_s ? (unsoftened_pc ? 0.0 : 0.5 * (ei2 + e2bar[v])) : e2c;
                or_pc_cell(xi, yi, zi, c, quad ? quad + 6 * v : NULL, ec, acc);
                cpc++;
            } else if (nchild[v] == 0) {
                for (int64_t j = first[v]; j < (int64_t)first[v] + count[v]; j++) {
                    if (j == i) continue;
                    const double ej = eps_s ? eps_s[j] : 0.0;
                    or_pp(xi, yi, zi, spos + 4 * j, eps_s ? 0.5 * (ei2 + ej * ej) : e2, acc);
                    cpp++;
                }
            } else {
                for (int ch = nchild[v] - 1; ch >= 0; ch--) stack[sp++] = child_first[v] + ch;
            }
        }
        const int64_t o = perm[i];
        for (int a = 0; a < 4; a++) out[4 * o + a] = acc[a];
        if (n_pp) n_pp[o] = cpp;
        if (n_pc) n_pc[o] = cpc;
        if (margin) margin[o] = mmin;
        if (a_abs) a_abs[o] = acc[4];
        free(stack);
    }
    return err;
}

/* ------------------------------------------------------------------------
 * The orbit loop around the force evaluation (Sec. 1: compute the forces,
 * integrate the orbits, repeat), as one leapfrog update per particle:
 *   v <- v + a dt_kick,   then   x <- x + v dt_drift   (the updated v).
 * A kick-drift-kick step of length dt is a kick by dt/2 with the forces at
 * the start, a drift by dt, new forces, and a kick by dt/2; the second half
 * kick and the next step's first half kick may be merged into one kick by dt.
 * pos, vel: n x 4 FP64, components 0..2 updated in place (3 untouched);
 * acc: n x 4 FP64 (ax, ay, az, phi).
 * ---------------------------------------------------------------------- */
void or_kick_drift(int64_t n, double* pos, double* vel, const double* acc, double dt_kick, double dt_drift)
{
    for (int64_t i = 0; i < n; i++) {
        for (int a = 0; a < 3; a++) {
            vel[4 * i + a] = vel[4 * i + a] + acc[4 * i + a] * dt_kick;
            pos[4 * i + a] = pos[4 * i + a] + vel[4 * i + a] * dt_drift;
        }
    }
}

/* One particle-cell term at target x (for the quadrupole pins). */
void or_pc_eval(const double* x, const double* com_m, const double* quad, double eps, double* out)
{
    double acc[5] = {0, 0, 0, 0, 0};
    or_pc(x[0], x[1], x[2], com_m, quad, eps * eps, acc);
    for (int a = 0; a < 4; a++) out[a] = acc[a];
}

/* ========================================================================
 * Learned opening criterion (an extension of Eq. 2's test, not in the paper).
 *
 * A small network predicts, for a (group, node) pair, log10 of the node's
 * relative force-error contribution; the node is accepted when the
 * prediction is below log10(tau) and a permissive geometric guard (Eq. 2 with
 * theta_max, applied to the group's box, node holding no member) passes.
 *
 * Features (all FP64 here):
 *   f1 = l / d            l = node cube side, d = |COM - group box centre|
 *   f2 = log10(M / M_tot)
 *   f3 = |I - (T/3) 1|_F / (M l^2)     (0 when no second moments)
 *   f4 = r_g / d          r_g = half diagonal of the group box
 *   f5 = level / 10
 *   f6 = log2(count) / 24
 * Network 6 -> 32 -> 32 -> 1, ReLU hidden layers; parameters packed as
 * W1[32][6], b1[32], W2[32][32], b2[32], W3[32], b3 (1313 values).
 * ====================================================================== */
#define OR_NF 6
#define OR_NH 32
#define OR_NPARAM (OR_NH * OR_NF + OR_NH + OR_NH * OR_NH + OR_NH + OR_NH + 1)

int or_mlp_nparams(void) { return OR_NPARAM; }

/* float -> bf16 -> float, round to nearest even (inference emulation) */
static double or_bf16(double x)
{
    float f = (float)x;
    uint32_t u;
    memcpy(&u, &f, 4);
    const uint32_t lsb = (u >> 16) & 1u;
    u += 0x7fffu + lsb;
    u &= 0xffff0000u;
    memcpy(&f, &u, 4);
    return f;
}

/* Forward pass of one sample; h1/h2 receive the hidden activations (after
 * ReLU) when non-NULL.  bf16 != 0 rounds inputs, weights and hidden
 * activations to bfloat16 as the in-walk inference does. */
static double or_mlp_one(const double* P, const double* x, int bf16, double* h1o, double* h2o)
{
    const double *W1 = P, *b1 = W1 + OR_NH * OR_NF, *W2 = b1 + OR_NH, *b2 = W2 + OR_NH * OR_NH,
                 *W3 = b2 + OR_NH, *b3 = W3 + OR_NH;
    double xin[OR_NF], h1[OR_NH], h2[OR_NH];
    for (int k = 0; k < OR_NF; k++) xin[k] = bf16 ? or_bf16(x[k]) : x[k];
    for (int j = 0; j < OR_NH; j++) {
        double s = b1[j];
        for (int k = 0; k < OR_NF; k++) s += (bf16 ? or_bf16(W1[j * OR_NF + k]) : W1[j * OR_NF + k]) * xin[k];
        h1[j] = s > 0 ? s : 0;
        if (bf16) h1[j] = or_bf16(h1[j]);
    }
    for (int j = 0; j < OR_NH; j++) {
        double s = b2[j];
        for (int k = 0; k < OR_NH; k++) s += (bf16 ? or_bf16(W2[j * OR_NH + k]) : W2[j * OR_NH + k]) * h1[k];
        h2[j] = s > 0 ? s : 0;
        if (bf16) h2[j] = or_bf16(h2[j]);
    }
    double y = b3[0];
    for (int k = 0; k < OR_NH; k++) y += (bf16 ? or_bf16(W3[k]) : W3[k]) * h2[k];
    if (h1o) memcpy(h1o, h1, sizeof(h1));
    if (h2o) memcpy(h2o, h2, sizeof(h2));
    return y;
}

void or_mlp_forward(const double* P, int64_t ns, const double* X, int bf16, double* y)
{
    int64_t i;
#pragma omp parallel for schedule(static)
    for (i = 0; i < ns; i++) y[i] = or_mlp_one(P, X + OR_NF * i, bf16, NULL, NULL);
}

/* Weighted mean squared error on log10 errors: w = under_weight when the
 * prediction is below the label (an under-predicted error is the unsafe
 * side), else 1.  Returns the loss; grad (OR_NPARAM) = d loss / d params. */
double or_mlp_loss_grad(const double* P, int64_t ns, const double* X, const double* Y, double under_weight,
                        double* grad)
{
    const double *W2 = P + OR_NH * OR_NF + OR_NH, *W3 = W2 + OR_NH * OR_NH + OR_NH;
    memset(grad, 0, sizeof(double) * OR_NPARAM);
    double* gW1 = grad;
    double* gb1 = gW1 + OR_NH * OR_NF;
    double* gW2 = gb1 + OR_NH;
    double* gb2 = gW2 + OR_NH * OR_NH;
    double* gW3 = gb2 + OR_NH;
    double* gb3 = gW3 + OR_NH;
    double loss = 0;
    for (int64_t i = 0; i < ns; i++) {
        double h1[OR_NH], h2[OR_NH];
        const double* x = X + OR_NF * i;
        const double yh = or_mlp_one(P, x, 0, h1, h2);
        const double r = yh - Y[i];
        const double w = (yh < Y[i]) ? under_weight : 1.0;
        loss += w * r * r;
        const double dy = 2.0 * w * r / (double)ns;
        gb3[0] += dy;
        double dh2[OR_NH], dh1[OR_NH];
        for (int k = 0; k < OR_NH; k++) {
            gW3[k] += dy * h2[k];
            dh2[k] = h2[k] > 0 ? dy * W3[k] : 0;
        }
        for (int k = 0; k < OR_NH; k++) dh1[k] = 0;
        for (int j = 0; j < OR_NH; j++) {
            gb2[j] += dh2[j];
            for (int k = 0; k < OR_NH; k++) {
                gW2[j * OR_NH + k] += dh2[j] * h1[k];
                dh1[k] += dh2[j] * W2[j * OR_NH + k];
            }
        }
        for (int j = 0; j < OR_NH; j++) {
            const double d1 = h1[j] > 0 ? dh1[j] : 0;
            gb1[j] += d1;
            for (int k = 0; k < OR_NF; k++) gW1[j * OR_NF + k] += d1 * x[k];
        }
    }
    return loss / (double)ns;
}

/* One Adam step (Kingma & Ba 2015) with bias correction; t counts from 1. */
void or_adam_step(int64_t np, double* P, const double* g, double* m, double* v, int64_t t, double lr, double b1,
                  double b2, double eps)
{
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t k = 0; k < np; k++) {
        m[k] = b1 * m[k] + (1 - b1) * g[k];
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k];
        P[k] -= lr * (m[k] / c1) / (sqrt(v[k] / c2) + eps);
    }
}

/* Features of (group box [lo, hi], node v); returns 0 when d == 0. */
static int or_mac_feat(const double* lo, const double* hi, const double* cm, const double* qd, double side,
                       int level, int count, double mtot, double* f)
{
    double c[3], r2 = 0, d2 = 0;
    for (int a = 0; a < 3; a++) {
        c[a] = 0.5 * (lo[a] + hi[a]);
        r2 += 0.25 * (hi[a] - lo[a]) * (hi[a] - lo[a]);
        d2 += (cm[a] - c[a]) * (cm[a] - c[a]);
    }
    const double d = sqrt(d2);
    if (!(d > 0)) return 0;
    double qn = 0;
    if (qd && cm[3] > 0) {
        const double T = qd[0] + qd[1] + qd[2];
        const double a0 = qd[0] - T / 3, a1 = qd[1] - T / 3, a2 = qd[2] - T / 3;
        qn = sqrt(a0 * a0 + a1 * a1 + a2 * a2 + 2 * (qd[3] * qd[3] + qd[4] * qd[4] + qd[5] * qd[5])) /
             (cm[3] * side * side);
    }
    f[0] = side / d;
    f[1] = (cm[3] > 0 && mtot > 0) ? log10(cm[3] / mtot) : -30.0;
    f[2] = qn;
    f[3] = sqrt(r2) / d;
    f[4] = level / 10.0;
    f[5] = log2((double)count) / 24.0;
    return 1;
}

/* Training pairs: for each listed group, the nodes accepted by the guard
 * alone (Eq. 2 with theta_guard via s_eff_guard, node holding no member),
 * their features, and the label log10(max over members of
 * |a_PC(node) - a_exact(node)| / |a_total,member|), a_PC with the given
 * order (quad may be NULL), a_exact the direct sum over the node's
 * particles.  a_tot: per Morton position, |a| of the member's total force.
 * The walk also descends into a guard-passing internal node whose label
 * exceeds descend_above (the network meets such nodes' children whenever it
 * rejects them), so the pairs cover every depth the network is asked about.
 * Returns the number of pairs written, or -1 if cap is exceeded. */
int64_t or_mac_training_pairs(const float* spos, int64_t nn, const int32_t* level, const int32_t* first,
                              const int32_t* count, const int32_t* child_first, const int32_t* nchild,
                              const double* com_m, const double* quad, const double* side,
                              const double* s_eff_guard, int64_t ng, const int32_t* gl_first,
                              const int32_t* gl_count, const double* a_tot, double eps, double descend_above,
                              int64_t cap, double* X, double* Y, int32_t* pair_group, int32_t* pair_node)
{
    const double e2 = eps * eps, mtot = com_m[3];
    int64_t np = 0;
    int32_t* stack = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
    if (!stack) return -1;
    for (int64_t g = 0; g < ng; g++) {
        const int64_t gb = gl_first[g], ge = gb + gl_count[g];
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) lo[a] = hi[a] = spos[4 * gb + a];
        for (int64_t k = gb; k < ge; k++)
            for (int a = 0; a < 3; a++) {
                const double v = spos[4 * k + a];
                if (v < lo[a]) lo[a] = v;
                if (v > hi[a]) hi[a] = v;
            }
        int64_t sp = 0;
        stack[sp++] = 0;
        while (sp > 0) {
            const int32_t v = stack[--sp];
            const double* c = com_m + 4 * v;
            double d2 = 0;
            for (int a = 0; a < 3; a++) {
                double t = 0;
                if (c[a] < lo[a]) t = lo[a] - c[a];
                else if (c[a] > hi[a]) t = c[a] - hi[a];
                d2 += t * t;
            }
            const int member = first[v] < ge && (int64_t)first[v] + count[v] > gb;
            if (d2 > s_eff_guard[v] && !member) {
                double f[OR_NF];
                if (!or_mac_feat(lo, hi, c, quad ? quad + 6 * v : NULL, side[v], level[v], count[v], mtot, f))
                    continue;
                double worst = 0;
                for (int64_t i = gb; i < ge; i++) {
                    const double xi = spos[4 * i], yi = spos[4 * i + 1], zi = spos[4 * i + 2];
                    double apc[5] = {0, 0, 0, 0, 0}, aex[5] = {0, 0, 0, 0, 0};
                    or_pc(xi, yi, zi, c, quad ? quad + 6 * v : NULL, e2, apc);
                    for (int64_t j = first[v]; j < (int64_t)first[v] + count[v]; j++)
                        or_pp(xi, yi, zi, spos + 4 * j, e2, aex);
                    const double dx = apc[0] - aex[0], dy = apc[1] - aex[1], dz = apc[2] - aex[2];
                    const double e = sqrt(dx * dx + dy * dy + dz * dz) / a_tot[i];
                    if (e > worst) worst = e;
                }
                if (np >= cap) {
                    free(stack);
                    return -1;
                }
                for (int k = 0; k < OR_NF; k++) X[OR_NF * np + k] = f[k];
                Y[np] = log10(worst > 1e-12 ? worst : 1e-12);
                pair_group[np] = (int32_t)g;
                pair_node[np] = v;
                np++;
                if (worst > descend_above && nchild[v] > 0)
                    for (int ch = nchild[v] - 1; ch >= 0; ch--) stack[sp++] = child_first[v] + ch;
            } else if (nchild[v] > 0) {
                for (int ch = nchild[v] - 1; ch >= 0; ch--) stack[sp++] = child_first[v] + ch;
            }
        }
    }
    free(stack);
    return np;
}

/* Group walk with the learned criterion.  A node passing the guard
 * (s_eff_guard, no member held) is accepted when the network's prediction
 * (bf16 inference emulation) is below log10(tau); when a feature lies outside
 * [fmin, fmax] the plain Eq. (2) test with theta_fb decides instead
 * (S_fb = (l/theta_fb + s)^2, s recovered from the guard's S_eff).
 * margin: per target, min over its group's network decisions of
 * |prediction - log10 tau| (infinity if none), and the guard margins. */
int or_force_groups_learned(int64_t n, const float* spos, const uint32_t* perm, int64_t nn, const int32_t* level,
                            const int32_t* first, const int32_t* count, const int32_t* child_first,
                            const int32_t* nchild, const double* com_m, const double* quad, const double* side,
                            const double* s_eff_guard, double theta_guard, double theta_fb, int64_t ng,
                            const int32_t* g_first, const int32_t* g_count, const uint8_t* group_mask,
                            const double* P, const double* fmin, const double* fmax, double tau, double eps,
                            double* out, double* margin_net, double* margin_geo, int64_t* n_pp, int64_t* n_pc)
{
    const double e2 = eps * eps, mtot = com_m[3], ltau = log10(tau);
    int err = 0;
    (void)n;
    int64_t g;
#pragma omp parallel for schedule(dynamic, 4)
    for (g = 0; g < ng; g++) {
        if (group_mask && !group_mask[g]) continue;
        const int64_t gb = g_first[g], ge = gb + g_count[g];
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) lo[a] = hi[a] = spos[4 * gb + a];
        for (int64_t k = gb; k < ge; k++)
            for (int a = 0; a < 3; a++) {
                const double v = spos[4 * k + a];
                if (v < lo[a]) lo[a] = v;
                if (v > hi[a]) hi[a] = v;
            }
        int32_t* stack = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
        int32_t* pc = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
        int32_t* pp = (int32_t*)malloc((size_t)nn * sizeof(int32_t));
        if (!stack || !pc || !pp) {
            free(stack); free(pc); free(pp);
#pragma omp atomic write
            err = -1;
            continue;
        }
        int64_t sp = 0, npc = 0, npp = 0;
        double mnet = INFINITY, mgeo = INFINITY;
        stack[sp++] = 0;
        while (sp > 0) {
            const int32_t v = stack[--sp];
            const double* c = com_m + 4 * v;
            double d2 = 0;
            for (int a = 0; a < 3; a++) {
                double t = 0;
                if (c[a] < lo[a]) t = lo[a] - c[a];
                else if (c[a] > hi[a]) t = c[a] - hi[a];
                d2 += t * t;
            }
            const int member = first[v] < ge && (int64_t)first[v] + count[v] > gb;
            int accept = 0;
            if (!member) {
                const double S = s_eff_guard[v];
                const double mg = fabs(d2 - S) / S;
                if (mg < mgeo) mgeo = mg;
                if (d2 > S) {
                    double f[OR_NF];
                    int inrange = or_mac_feat(lo, hi, c, quad ? quad + 6 * v : NULL, side[v], level[v], count[v],
                                              mtot, f);
                    for (int k = 0; inrange && k < OR_NF; k++)
                        if (f[k] < fmin[k] || f[k] > fmax[k]) inrange = 0;
                    if (inrange) {
                        const double yh = or_mlp_one(P, f, 1, NULL, NULL);
                        const double mn = fabs(yh - ltau);
                        if (mn < mnet) mnet = mn;
                        accept = yh < ltau;
                    } else {
                        const double s = sqrt(S) - side[v] / theta_guard;
                        const double t = side[v] / theta_fb + (s > 0 ? s : 0);
                        const double Sf = t * t;
                        const double mf = fabs(d2 - Sf) / Sf;
                        if (mf < mgeo) mgeo = mf;
                        accept = d2 > Sf;
                    }
                }
            }
            if (accept) pc[npc++] = v;
            else if (nchild[v] == 0) pp[npp++] = v;
            else
                for (int ch = nchild[v] - 1; ch >= 0; ch--) stack[sp++] = child_first[v] + ch;
        }
        for (int64_t i = gb; i < ge; i++) {
            const double xi = spos[4 * i], yi = spos[4 * i + 1], zi = spos[4 * i + 2];
            double acc[5] = {0, 0, 0, 0, 0};
            int64_t cnt_pp = 0;
            for (int64_t t = 0; t < npc; t++)
                or_pc_cell(xi, yi, zi, com_m + 4 * pc[t], quad ? quad + 6 * pc[t] : NULL, e2, acc);
            for (int64_t t = 0; t < npp; t++)
                for (int64_t j = first[pp[t]]; j < (int64_t)first[pp[t]] + count[pp[t]]; j++) {
                    if (j == i) continue;
                    or_pp(xi, yi, zi, spos + 4 * j, e2, acc);
                    cnt_pp++;
                }
            const int64_t o = perm[i];
            for (int a = 0; a < 4; a++) out[4 * o + a] = acc[a];
            if (margin_net) margin_net[o] = mnet;
            if (margin_geo) margin_geo[o] = mgeo;
            if (n_pp) n_pp[o] = cnt_pp;
            if (n_pc) n_pc[o] = npc;
        }
        free(stack);
        free(pc);
        free(pp);
    }
    return err;
}

/* Features of one (group box, node) pair (for the feature pins). */
int or_mac_features_one(const double* lo, const double* hi, const double* cm, const double* qd, double side,
                        int level, int count, double mtot, double* f)
{
    return or_mac_feat(lo, hi, cm, qd, side, level, count, mtot, f);
}

/* ========================================================================
 * Neighbour search, the short-range application of the general tree walk
 * (Sec. 4.3, Fig. 4), here by its plain definition (all pairs).
 *
 * For particle i with search radius h_i, particle j != i is a neighbour when
 * |x_j - x_i| < h_i, the decision taken in FP32 as the device takes it:
 * d = x_j - x_i per axis (FP32), r2 = fma(dz, dz, fma(dy, dy, dx * dx)),
 * neighbour iff r2 < h_i * h_i (FP32 product).  The SPH density
 *   rho_i = sum over i itself and its neighbours of m_j W(r_ij, h_i)
 * uses the cubic spline of Monaghan & Lattanzio (1985) with support h:
 *   W(r, h) = 8 / (pi h^3) * { 1 - 6 q^2 + 6 q^3,  0 <= q <= 1/2
 *                              2 (1 - q)^3,        1/2 < q <= 1 },  q = r / h
 * (normalised: its integral over space is 1), in FP64 with r = sqrt(r2) from
 * the FP32 r2 above.  count[i] excludes i itself.
 * ---------------------------------------------------------------------- */
double or_sph_kernel(double r, double h)
{
    const double q = r / h;
    const double c = 8.0 / (M_PI * h * h * h);
    if (q <= 0.5) return c * (1.0 - 6.0 * q * q + 6.0 * q * q * q);
    if (q <= 1.0) return c * 2.0 * (1.0 - q) * (1.0 - q) * (1.0 - q);
    return 0.0;
}

void or_sph_density(int64_t n, const float* pos, const float* h, int32_t* count, double* rho)
{
    int64_t i;
#pragma omp parallel for schedule(dynamic, 16)
    for (i = 0; i < n; i++) {
        const float xi = pos[4 * i], yi = pos[4 * i + 1], zi = pos[4 * i + 2];
        const float hi = h[i];
        const float h2 = hi * hi;
        double r = (double)pos[4 * i + 3] * or_sph_kernel(0.0, hi);
        int32_t c = 0;
        for (int64_t j = 0; j < n; j++) {
            if (j == i) continue;
            const float dx = pos[4 * j] - xi, dy = pos[4 * j + 1] - yi, dz = pos[4 * j + 2] - zi;
            const float r2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
            if (r2 < h2) {
                c++;
                r += (double)pos[4 * j + 3] * or_sph_kernel(sqrt((double)r2), hi);
            }
        }
        count[i] = c;
        rho[i] = r;
    }
}
