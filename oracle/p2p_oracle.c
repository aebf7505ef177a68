/*
 * Plain FP64 CPU oracle for the near-field P2P operator of MLFMA.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent reference that the
 * CUDA library is checked against.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may load it.  It shares no code,
 * header, table or helper with the CUDA path, and the CUDA path never calls it.
 *
 * What it computes (Sec. 3.1 tree of leaf boxes, Sec. 3.2 indexing method and
 * Sec. 3.3 repetition method, which are two data layouts of the same sum; the
 * CPU baseline of Sec. 4.1 traverses boxes in Morton order and, for every
 * target, visits the sources of the neighbouring boxes once):
 *
 *   cell_a(x) = clamp(floor((x_a - lo_a) / h), 0, ng-1)        a = x, y, z
 *   key(x)    = Morton interleave of (cx, cy, cz), x at bit 0, y at bit 1,
 *               z at bit 2 of every bit triple (21 bits per axis)
 *   box(x)    = rank of key(x) among the distinct keys of the point set
 *   nbr(b)    = boxes b' whose cells are within Chebyshev distance 1 of b's
 *               cell (own box included, no periodic wrap), ascending id
 *   out_i     = sum over j with box(j) in nbr(box(i)) and r_ij > 0 of
 *               G(r_ij) * lambda_j
 *
 *   Helmholtz:  G(r) = exp(+i k r) / (4 pi r)
 *   Laplace:    G(r) = 1 / (4 pi r)
 *
 * The same sum between two point sets -- targets x_i and sources y_j binned on
 * one grid, the neighbours of a target box being the source boxes around its
 * cell -- is oracle_p2p_st at the end of this file (Sec. 3.1 keeps target and
 * source coordinates as separate arrays).
 *
 * The paper's own test kernel is a 2D electric potential whose formula it
 * never prints (Sec. 2 and Sec. 4); the 3D Helmholtz / Laplace kernels and the
 * 27-box neighbourhood (the 3D analogue of the 9 boxes of Sec. 3.2) are the
 * readings this build takes.  Every computation is plain IEEE double: the cell
 * index uses one subtraction and one division (no fused multiply-add), so a
 * GPU that performs the same two double operations gets the same cell.
 *
 * Loop order: boxes in id order -> targets of the box in sorted order ->
 * neighbour boxes in ascending id -> sources of that box in sorted order.
 * Points inside one box keep their original relative order (stable sort on
 * (key, original index)).
 *
 * Compile with -O2 -fno-fast-math -ffp-contract=off.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORACLE_PI 3.14159265358979323846

enum { OK = 0, ERR_INVALID = 1, ERR_ALLOC = 2 };
enum { K_HELMHOLTZ = 0, K_LAPLACE = 1 };

/* ---------------------------------------------------------------- cells ---- */

static int64_t morton_interleave(int64_t cx, int64_t cy, int64_t cz) {
    int64_t key = 0;
    for (int bit = 0; bit < 21; ++bit) {
        key |= ((cx >> bit) & 1) << (3 * bit);
        key |= ((cy >> bit) & 1) << (3 * bit + 1);
        key |= ((cz >> bit) & 1) << (3 * bit + 2);
    }
    return key;
}

static void morton_split(int64_t key, int64_t cell[3]) {
    cell[0] = cell[1] = cell[2] = 0;
    for (int bit = 0; bit < 21; ++bit) {
        cell[0] |= ((key >> (3 * bit)) & 1) << bit;
        cell[1] |= ((key >> (3 * bit + 1)) & 1) << bit;
        cell[2] |= ((key >> (3 * bit + 2)) & 1) << bit;
    }
}

static int64_t cell_index(double x, double lo, double h, int32_t ng) {
    double t = (x - lo) / h;
    double f = floor(t);
    if (f < 0.0) f = 0.0;
    if (f > (double)(ng - 1)) f = (double)(ng - 1);
    return (int64_t)f;
}

int oracle_morton_key(int64_t cx, int64_t cy, int64_t cz, int64_t* key) {
    if (cx < 0 || cy < 0 || cz < 0 || cx >= (1 << 21) || cy >= (1 << 21) || cz >= (1 << 21))
        return ERR_INVALID;
    *key = morton_interleave(cx, cy, cz);
    return OK;
}

int oracle_point_cells(const double* pts, int64_t n, const double lo[3], double h, int32_t ng,
                       int64_t* cells /* n x 3 */) {
    if (n < 0 || !(h > 0.0) || ng < 1 || ng > (1 << 21)) return ERR_INVALID;
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double x = pts[3 * i + a];
            if (!isfinite(x)) return ERR_INVALID;
            cells[3 * i + a] = cell_index(x, lo[a], h, ng);
        }
    return OK;
}

/* -------------------------------------------------------------- binning ---- */

typedef struct {
    int64_t key;
    int64_t idx;
} keyed_point;

static int cmp_keyed(const void* a, const void* b) {
    const keyed_point* p = (const keyed_point*)a;
    const keyed_point* q = (const keyed_point*)b;
    if (p->key != q->key) return p->key < q->key ? -1 : 1;
    if (p->idx != q->idx) return p->idx < q->idx ? -1 : 1;
    return 0;
}

/*
 * Leaf binning.  perm[s] = original index of the s-th point in box order,
 * point_box[i] = box id of original point i, box_keys[b] = Morton key of box
 * b, box_ptr[b] .. box_ptr[b+1] = the sorted positions of box b's points.
 * box_keys and box_ptr must hold n and n+1 entries.
 */
int oracle_bin(const double* pts, int64_t n, const double lo[3], double h, int32_t ng,
               int32_t* perm, int32_t* point_box, int64_t* box_keys, int32_t* box_ptr,
               int32_t* num_boxes) {
    if (n < 0 || n > INT32_MAX - 1 || !(h > 0.0) || ng < 1 || ng > (1 << 21)) return ERR_INVALID;
    *num_boxes = 0;
    box_ptr[0] = 0;
    if (n == 0) return OK;
    keyed_point* kp = (keyed_point*)malloc(sizeof(keyed_point) * (size_t)n);
    if (!kp) return ERR_ALLOC;
    for (int64_t i = 0; i < n; ++i) {
        int64_t c[3];
        for (int a = 0; a < 3; ++a) {
            double x = pts[3 * i + a];
            if (!isfinite(x)) {
                free(kp);
                return ERR_INVALID;
            }
            c[a] = cell_index(x, lo[a], h, ng);
        }
        kp[i].key = morton_interleave(c[0], c[1], c[2]);
        kp[i].idx = i;
    }
    qsort(kp, (size_t)n, sizeof(keyed_point), cmp_keyed);
    int32_t nb = 0;
    for (int64_t s = 0; s < n; ++s) {
        if (s == 0 || kp[s].key != kp[s - 1].key) {
            box_keys[nb] = kp[s].key;
            box_ptr[nb] = (int32_t)s;
            ++nb;
        }
        perm[s] = (int32_t)kp[s].idx;
        point_box[kp[s].idx] = nb - 1;
    }
    box_ptr[nb] = (int32_t)n;
    *num_boxes = nb;
    free(kp);
    return OK;
}

/* ------------------------------------------------------------ neighbours --- */

static int32_t find_box(const int64_t* keys, int32_t nb, int64_t key) {
    int32_t lo = 0, hi = nb - 1;
    while (lo <= hi) {
        int32_t mid = lo + (hi - lo) / 2;
        if (keys[mid] == key) return mid;
        if (keys[mid] < key) lo = mid + 1;
        else hi = mid - 1;
    }
    return -1;
}

/* nbr_ptr holds num_boxes+1 entries, nbr_idx up to 27*num_boxes entries. */
int oracle_neighbors(const int64_t* box_keys, int32_t nb, int32_t ng, int32_t* nbr_ptr,
                     int32_t* nbr_idx) {
    if (nb < 0 || ng < 1 || ng > (1 << 21)) return ERR_INVALID;
    int64_t nnz = 0;
    nbr_ptr[0] = 0;
    for (int32_t b = 0; b < nb; ++b) {
        int64_t c[3];
        morton_split(box_keys[b], c);
        int32_t found[27];
        int nf = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= ng || y >= ng || z >= ng) continue;
                    int32_t id = find_box(box_keys, nb, morton_interleave(x, y, z));
                    if (id >= 0) found[nf++] = id;
                }
        /* ascending box id */
        for (int a = 1; a < nf; ++a) {
            int32_t v = found[a];
            int q = a - 1;
            while (q >= 0 && found[q] > v) {
                found[q + 1] = found[q];
                --q;
            }
            found[q + 1] = v;
        }
        for (int a = 0; a < nf; ++a) nbr_idx[nnz++] = found[a];
        nbr_ptr[b + 1] = (int32_t)nnz;
    }
    return OK;
}

/* --------------------------------------------------------------- kernels --- */

/* G(r) for r > 0; conj = 1 gives the complex conjugate exp(-ikr)/(4 pi r). */
static void green(int kernel, double k, int conj, double r, double* gr, double* gi) {
    double a = 1.0 / (4.0 * ORACLE_PI * r);
    if (kernel == K_LAPLACE) {
        *gr = a;
        *gi = 0.0;
        return;
    }
    double kr = k * r;
    *gr = cos(kr) * a;
    *gi = (conj ? -sin(kr) : sin(kr)) * a;
}

/* dG/dr for r > 0: Helmholtz exp(ikr)(ikr - 1)/(4 pi r^2), Laplace -1/(4 pi r^2). */
static void green_dr(int kernel, double k, double r, double* dr, double* di) {
    double a = 1.0 / (4.0 * ORACLE_PI * r * r);
    if (kernel == K_LAPLACE) {
        *dr = -a;
        *di = 0.0;
        return;
    }
    double kr = k * r, c = cos(kr), s = sin(kr);
    /* (c + i s)(-1 + i kr) = (-c - s kr) + i (c kr - s) */
    *dr = (-c - s * kr) * a;
    *di = (c * kr - s) * a;
}

typedef struct {
    int64_t n;
    int32_t nb;
    int32_t* perm;
    int32_t* point_box;
    int64_t* box_keys;
    int32_t* box_ptr;
    int32_t* nbr_ptr;
    int32_t* nbr_idx;
} tree;

static void tree_free(tree* t) {
    free(t->perm);
    free(t->point_box);
    free(t->box_keys);
    free(t->box_ptr);
    free(t->nbr_ptr);
    free(t->nbr_idx);
}

static int tree_build(const double* pts, int64_t n, const double lo[3], double h, int32_t ng, tree* t) {
    memset(t, 0, sizeof(*t));
    t->n = n;
    size_t m = (size_t)(n > 0 ? n : 1);
    t->perm = (int32_t*)malloc(sizeof(int32_t) * m);
    t->point_box = (int32_t*)malloc(sizeof(int32_t) * m);
    t->box_keys = (int64_t*)malloc(sizeof(int64_t) * m);
    t->box_ptr = (int32_t*)malloc(sizeof(int32_t) * (m + 1));
    t->nbr_ptr = (int32_t*)malloc(sizeof(int32_t) * (m + 1));
    t->nbr_idx = (int32_t*)malloc(sizeof(int32_t) * 27 * m);
    if (!t->perm || !t->point_box || !t->box_keys || !t->box_ptr || !t->nbr_ptr || !t->nbr_idx) {
        tree_free(t);
        return ERR_ALLOC;
    }
    int st = oracle_bin(pts, n, lo, h, ng, t->perm, t->point_box, t->box_keys, t->box_ptr, &t->nb);
    if (st == OK) st = oracle_neighbors(t->box_keys, t->nb, ng, t->nbr_ptr, t->nbr_idx);
    if (st != OK) tree_free(t);
    return st;
}

/* Sum for one target (original index i) over its neighbourhood, all RHS. */
static void target_sum(const tree* t, const double* pts, int kernel, double k, int conj,
                       const double* lam, int32_t nrhs, int64_t i, double* out /* nrhs x 2 */) {
    for (int32_t q = 0; q < nrhs; ++q) out[2 * q] = out[2 * q + 1] = 0.0;
    int32_t b = t->point_box[i];
    const double* xi = pts + 3 * i;
    for (int32_t e = t->nbr_ptr[b]; e < t->nbr_ptr[b + 1]; ++e) {
        int32_t nbx = t->nbr_idx[e];
        for (int32_t s = t->box_ptr[nbx]; s < t->box_ptr[nbx + 1]; ++s) {
            int64_t j = t->perm[s];
            const double* xj = pts + 3 * j;
            double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue; /* r = 0: self pair or duplicate point */
            double gr, gi;
            green(kernel, k, conj, sqrt(r2), &gr, &gi);
            const double* lj = lam + 2 * (size_t)nrhs * (size_t)j;
            for (int32_t q = 0; q < nrhs; ++q) {
                double lr = lj[2 * q], li = lj[2 * q + 1];
                out[2 * q] += gr * lr - gi * li;
                out[2 * q + 1] += gr * li + gi * lr;
            }
        }
    }
}

/*
 * out = A lambda (conj = 0) or conj(A) lambda (conj = 1; since A is complex
 * symmetric, conj(A) = A^H, the adjoint).  pts: n x 3 doubles; lam and out:
 * n x nrhs complex as interleaved (re, im) doubles, original point order.
 */
int oracle_p2p(const double* pts, int64_t n, const double lo[3], double h, int32_t ng, int kernel,
               double k, int conj, const double* lam, int32_t nrhs, double* out) {
    if (nrhs < 1 || (kernel != K_HELMHOLTZ && kernel != K_LAPLACE)) return ERR_INVALID;
    tree t;
    int st = tree_build(pts, n, lo, h, ng, &t);
    if (st != OK) return st;
    for (int32_t b = 0; b < t.nb; ++b)
        for (int32_t s = t.box_ptr[b]; s < t.box_ptr[b + 1]; ++s) {
            int64_t i = t.perm[s];
            target_sum(&t, pts, kernel, k, conj, lam, nrhs, i, out + 2 * (size_t)nrhs * (size_t)i);
        }
    tree_free(&t);
    return OK;
}

/* The same sum for a list of targets only (original indices); out: nt x nrhs complex. */
int oracle_p2p_targets(const double* pts, int64_t n, const double lo[3], double h, int32_t ng,
                       int kernel, double k, int conj, const double* lam, int32_t nrhs,
                       const int64_t* targets, int64_t nt, double* out) {
    if (nrhs < 1 || (kernel != K_HELMHOLTZ && kernel != K_LAPLACE)) return ERR_INVALID;
    for (int64_t a = 0; a < nt; ++a)
        if (targets[a] < 0 || targets[a] >= n) return ERR_INVALID;
    tree t;
    int st = tree_build(pts, n, lo, h, ng, &t);
    if (st != OK) return st;
    for (int64_t a = 0; a < nt; ++a)
        target_sum(&t, pts, kernel, k, conj, lam, nrhs, targets[a], out + 2 * (size_t)nrhs * (size_t)a);
    tree_free(&t);
    return OK;
}

/* Number of ordered (target, source) pairs with r > 0 in the neighbourhoods. */
int oracle_pair_count(const double* pts, int64_t n, const double lo[3], double h, int32_t ng,
                      int64_t* pairs) {
    tree t;
    int st = tree_build(pts, n, lo, h, ng, &t);
    if (st != OK) return st;
    int64_t p = 0;
    for (int64_t i = 0; i < n; ++i) {
        int32_t b = t.point_box[i];
        const double* xi = pts + 3 * i;
        for (int32_t e = t.nbr_ptr[b]; e < t.nbr_ptr[b + 1]; ++e) {
            int32_t nbx = t.nbr_idx[e];
            for (int32_t s = t.box_ptr[nbx]; s < t.box_ptr[nbx + 1]; ++s) {
                const double* xj = pts + 3 * (int64_t)t.perm[s];
                double dx = xi[0] - xj[0], dy = xi[1] - xj[1], dz = xi[2] - xj[2];
                if (dx * dx + dy * dy + dz * dz != 0.0) ++p;
            }
        }
    }
    *pairs = p;
    tree_free(&t);
    return OK;
}

/*
 * Gradient of a real loss L with respect to the point coordinates, given the
 * upstream gradient g = dL/dRe(out) + i dL/dIm(out) of out = A lambda, with
 * the box structure held fixed.  With dr_mj = (x_m - x_j).(dx_m - dx_j)/r:
 *
 *   dL/dx_m = sum_{j in nbr(m), r > 0} sum_q
 *             Re[ G'(r_mj) (conj(g_mq) lambda_jq + conj(g_jq) lambda_mq) ] (x_m - x_j) / r_mj
 *
 * grad: n x 3 doubles in original order.
 */
int oracle_grad_points(const double* pts, int64_t n, const double lo[3], double h, int32_t ng,
                       int kernel, double k, const double* lam, const double* g, int32_t nrhs,
                       double* grad) {
    if (nrhs < 1 || (kernel != K_HELMHOLTZ && kernel != K_LAPLACE)) return ERR_INVALID;
    tree t;
    int st = tree_build(pts, n, lo, h, ng, &t);
    if (st != OK) return st;
    for (int64_t m = 0; m < n; ++m) {
        double acc[3] = {0.0, 0.0, 0.0};
        int32_t b = t.point_box[m];
        const double* xm = pts + 3 * m;
        const double* lm = lam + 2 * (size_t)nrhs * (size_t)m;
        const double* gm = g + 2 * (size_t)nrhs * (size_t)m;
        for (int32_t e = t.nbr_ptr[b]; e < t.nbr_ptr[b + 1]; ++e) {
            int32_t nbx = t.nbr_idx[e];
            for (int32_t s = t.box_ptr[nbx]; s < t.box_ptr[nbx + 1]; ++s) {
                int64_t j = t.perm[s];
                const double* xj = pts + 3 * j;
                double d[3] = {xm[0] - xj[0], xm[1] - xj[1], xm[2] - xj[2]};
                double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                if (r2 == 0.0) continue;
                double r = sqrt(r2);
                double dgr, dgi;
                green_dr(kernel, k, r, &dgr, &dgi);
                const double* lj = lam + 2 * (size_t)nrhs * (size_t)j;
                const double* gj = g + 2 * (size_t)nrhs * (size_t)j;
                double w = 0.0;
                for (int32_t q = 0; q < nrhs; ++q) {
                    /* c = conj(g_m) lambda_j + conj(g_j) lambda_m */
                    double cr = gm[2 * q] * lj[2 * q] + gm[2 * q + 1] * lj[2 * q + 1] +
                                gj[2 * q] * lm[2 * q] + gj[2 * q + 1] * lm[2 * q + 1];
                    double ci = gm[2 * q] * lj[2 * q + 1] - gm[2 * q + 1] * lj[2 * q] +
                                gj[2 * q] * lm[2 * q + 1] - gj[2 * q + 1] * lm[2 * q];
                    w += dgr * cr - dgi * ci; /* Re(G' c) */
                }
                for (int a = 0; a < 3; ++a) acc[a] += w * d[a] / r;
            }
        }
        for (int a = 0; a < 3; ++a) grad[3 * m + a] = acc[a];
    }
    tree_free(&t);
    return OK;
}

/* ------------------------------------------- separate targets and sources --- */
/*
 * The paper's tree object keeps target and source coordinates as separate
 * arrays (Sec. 3.1; Sec. 3.2 lists the target coordinates and the source
 * coordinates of each box separately).  Here both sets are binned on the same
 * uniform leaf grid, each with its own Morton-ranked box ids; the neighbours of
 * target box b are the non-empty SOURCE boxes whose cells lie within Chebyshev
 * distance 1 of b's cell, ascending source box id; a target and a source at
 * the same position (r = 0) are skipped, as for one point set.
 *
 *   out_i = sum over sources j with cell(j) within distance 1 of cell(i), r_ij > 0, of G(r_ij) lambda_j
 *
 * Loop order: target boxes in id order -> targets of the box in sorted order ->
 * neighbour source boxes ascending -> sources of that box in sorted order.
 */

/* nbr_ptr: nbt + 1 entries; nbr_idx: up to 27 * nbt entries. */
int oracle_neighbors_st(const int64_t* tgt_keys, int32_t nbt, const int64_t* src_keys, int32_t nbs, int32_t ng,
                        int32_t* nbr_ptr, int32_t* nbr_idx) {
    if (nbt < 0 || nbs < 0 || ng < 1 || ng > (1 << 21)) return ERR_INVALID;
    int64_t nnz = 0;
    nbr_ptr[0] = 0;
    for (int32_t b = 0; b < nbt; ++b) {
        int64_t c[3];
        morton_split(tgt_keys[b], c);
        int32_t found[27];
        int nf = 0;
        for (int dz = -1; dz <= 1; ++dz)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int64_t x = c[0] + dx, y = c[1] + dy, z = c[2] + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= ng || y >= ng || z >= ng) continue;
                    int32_t id = find_box(src_keys, nbs, morton_interleave(x, y, z));
                    if (id >= 0) found[nf++] = id;
                }
        for (int a = 1; a < nf; ++a) {
            int32_t v = found[a];
            int q = a - 1;
            while (q >= 0 && found[q] > v) {
                found[q + 1] = found[q];
                --q;
            }
            found[q + 1] = v;
        }
        for (int a = 0; a < nf; ++a) nbr_idx[nnz++] = found[a];
        nbr_ptr[b + 1] = (int32_t)nnz;
    }
    return OK;
}

typedef struct {
    tree t;     /* targets: binning, point_box, box_keys, box_ptr (nbr_* unused) */
    tree s;     /* sources: binning */
    int32_t* nbr_ptr;
    int32_t* nbr_idx;
} tree_st;

static void tree_st_free(tree_st* q) {
    tree_free(&q->t);
    tree_free(&q->s);
    free(q->nbr_ptr);
    free(q->nbr_idx);
}

static int bin_only(const double* pts, int64_t n, const double lo[3], double h, int32_t ng, tree* t) {
    memset(t, 0, sizeof(*t));
    t->n = n;
    size_t m = (size_t)(n > 0 ? n : 1);
    t->perm = (int32_t*)malloc(sizeof(int32_t) * m);
    t->point_box = (int32_t*)malloc(sizeof(int32_t) * m);
    t->box_keys = (int64_t*)malloc(sizeof(int64_t) * m);
    t->box_ptr = (int32_t*)malloc(sizeof(int32_t) * (m + 1));
    if (!t->perm || !t->point_box || !t->box_keys || !t->box_ptr) {
        tree_free(t);
        return ERR_ALLOC;
    }
    int st = oracle_bin(pts, n, lo, h, ng, t->perm, t->point_box, t->box_keys, t->box_ptr, &t->nb);
    if (st != OK) tree_free(t);
    return st;
}

static int tree_st_build(const double* tgt, int64_t nt, const double* src, int64_t ns, const double lo[3], double h,
                         int32_t ng, tree_st* q) {
    memset(q, 0, sizeof(*q));
    int st = bin_only(tgt, nt, lo, h, ng, &q->t);
    if (st != OK) return st;
    st = bin_only(src, ns, lo, h, ng, &q->s);
    if (st != OK) {
        tree_free(&q->t);
        return st;
    }
    size_t mb = (size_t)(q->t.nb > 0 ? q->t.nb : 1);
    q->nbr_ptr = (int32_t*)malloc(sizeof(int32_t) * (mb + 1));
    q->nbr_idx = (int32_t*)malloc(sizeof(int32_t) * 27 * mb);
    if (!q->nbr_ptr || !q->nbr_idx) {
        tree_st_free(q);
        return ERR_ALLOC;
    }
    st = oracle_neighbors_st(q->t.box_keys, q->t.nb, q->s.box_keys, q->s.nb, ng, q->nbr_ptr, q->nbr_idx);
    if (st != OK) tree_st_free(q);
    return st;
}

/* Sum for one target (original index i of the target set) over the sources of its neighbourhood. */
static void target_sum_st(const tree_st* q, const double* tgt, const double* src, int kernel, double k, int conj,
                          const double* lam, int32_t nrhs, int64_t i, double* out) {
    for (int32_t r = 0; r < nrhs; ++r) out[2 * r] = out[2 * r + 1] = 0.0;
    int32_t b = q->t.point_box[i];
    const double* xi = tgt + 3 * i;
    for (int32_t e = q->nbr_ptr[b]; e < q->nbr_ptr[b + 1]; ++e) {
        int32_t c = q->nbr_idx[e];
        for (int32_t s = q->s.box_ptr[c]; s < q->s.box_ptr[c + 1]; ++s) {
            int64_t j = q->s.perm[s];
            const double* yj = src + 3 * j;
            double dx = xi[0] - yj[0], dy = xi[1] - yj[1], dz = xi[2] - yj[2];
            double r2 = dx * dx + dy * dy + dz * dz;
            if (r2 == 0.0) continue; /* a target at a source's position */
            double gr, gi;
            green(kernel, k, conj, sqrt(r2), &gr, &gi);
            const double* lj = lam + 2 * (size_t)nrhs * (size_t)j;
            for (int32_t r = 0; r < nrhs; ++r) {
                double lr = lj[2 * r], li = lj[2 * r + 1];
                out[2 * r] += gr * lr - gi * li;
                out[2 * r + 1] += gr * li + gi * lr;
            }
        }
    }
}

/*
 * out (nt x nrhs complex, target order) = A lambda with A the nt x ns near-field
 * operator from the sources to the targets; conj = 1 gives conj(A) lambda.
 * lam: ns x nrhs complex (source order).  The adjoint A^H g (source space) is
 * the same call with the roles of the two sets exchanged and conj = 1, since
 * G(x, y) = G(y, x) and the neighbour relation is symmetric.
 */
int oracle_p2p_st(const double* tgt, int64_t nt, const double* src, int64_t ns, const double lo[3], double h,
                  int32_t ng, int kernel, double k, int conj, const double* lam, int32_t nrhs, double* out) {
    if (nrhs < 1 || (kernel != K_HELMHOLTZ && kernel != K_LAPLACE)) return ERR_INVALID;
    tree_st q;
    int st = tree_st_build(tgt, nt, src, ns, lo, h, ng, &q);
    if (st != OK) return st;
    for (int32_t b = 0; b < q.t.nb; ++b)
        for (int32_t s = q.t.box_ptr[b]; s < q.t.box_ptr[b + 1]; ++s) {
            int64_t i = q.t.perm[s];
            target_sum_st(&q, tgt, src, kernel, k, conj, lam, nrhs, i, out + 2 * (size_t)nrhs * (size_t)i);
        }
    tree_st_free(&q);
    return OK;
}

/* The same sum for a list of targets (original target indices) only; out: count x nrhs complex. */
int oracle_p2p_st_targets(const double* tgt, int64_t nt, const double* src, int64_t ns, const double lo[3],
                          double h, int32_t ng, int kernel, double k, int conj, const double* lam, int32_t nrhs,
                          const int64_t* targets, int64_t count, double* out) {
    if (nrhs < 1 || (kernel != K_HELMHOLTZ && kernel != K_LAPLACE)) return ERR_INVALID;
    for (int64_t a = 0; a < count; ++a)
        if (targets[a] < 0 || targets[a] >= nt) return ERR_INVALID;
    tree_st q;
    int st = tree_st_build(tgt, nt, src, ns, lo, h, ng, &q);
    if (st != OK) return st;
    for (int64_t a = 0; a < count; ++a)
        target_sum_st(&q, tgt, src, kernel, k, conj, lam, nrhs, targets[a], out + 2 * (size_t)nrhs * (size_t)a);
    tree_st_free(&q);
    return OK;
}
