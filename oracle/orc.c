/*
 * Oracle (test infrastructure only): plain, slow CPU reference for the Sylvester inertia count.
 *
 * Only tests, the smoke check and the benchmark's CPU-baseline leg may load this file's library.
 * It shares no code, header or table with the GPU path.
 *
 * What it computes.  For the pencil (A, B) and a shift sigma, nu_sigma(A, B) is the number of
 * eigenvalues of A x = lambda B x below sigma (Section 2.1).  By Sylvester's law of inertia it equals
 * the number of negative eigenvalues of the block-diagonal D of any factorization
 * P (A - sigma B) P^T = L D L^T (Algorithm 1, the nu_0(D, I) step).  Two plain routes are here:
 *
 *  (c1) orc_dense_bk: unblocked Bunch-Kaufman LDL^T with partial pivoting on a dense symmetric
 *       matrix (the stability permutation P the paper cites [Bunch-Kaufman 1977]),
 *       alpha = (1 + sqrt(17)) / 8.
 *  (c3) orc_sparse_inertia: a plain multifrontal sparse LDL^T of A - sigma B with its own
 *       fill-reducing nested-dissection ordering Q (Algorithm 1', the PQ(A - sigma B)Q^T P^T step),
 *       dense fronts, pivoting restricted to each front's fully-summed block with a threshold test,
 *       and pivots that fail it passed to the parent front.
 *
 * Sign rule for a 2x2 block [a b; b c] of D (the paper only says "negative eigenvalues of D"):
 * det < 0 -> one negative, one positive; det > 0 -> two of the sign of a + c;
 * det == 0 -> one zero and one of the sign of a + c (two zeros if a + c == 0).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define BK_ALPHA 0.6403882032022076 /* (1 + sqrt(17)) / 8 */

typedef struct { int64_t neg, zero, pos, delayed, n2x2; } orc_inertia;

static void count_1x1(double d, orc_inertia *in) {
  if (d < 0) in->neg++; else if (d > 0) in->pos++; else in->zero++;
}

static void count_2x2(double a, double b, double c, orc_inertia *in) {
  double det = a * c - b * b, tr = a + c;
  in->n2x2++;
  if (det < 0) { in->neg++; in->pos++; return; }
  if (det > 0) { if (tr < 0) in->neg += 2; else in->pos += 2; return; }
  if (tr < 0) { in->neg++; in->zero++; } else if (tr > 0) { in->pos++; in->zero++; } else in->zero += 2;
}

/* Element (i, j) of a symmetric matrix held in the lower triangle of column-major storage. */
#define LO(M, ld, i, j) ((i) >= (j) ? (M)[(size_t)(j) * (ld) + (i)] : (M)[(size_t)(i) * (ld) + (j)])

/* Symmetric interchange of indices p < q in lower storage, over the trailing rows/cols >= 0.
 * Columns 0..p-1 are swapped too (rows p and q of the already computed L). */
static void sym_swap(double *M, int64_t ld, int64_t m, int64_t p, int64_t q) {
  if (p == q) return;
  if (p > q) { int64_t t = p; p = q; q = t; }
  for (int64_t j = 0; j < p; ++j) {           /* rows p and q of earlier columns */
    double t = M[j * ld + p]; M[j * ld + p] = M[j * ld + q]; M[j * ld + q] = t;
  }
  { double t = M[p * ld + p]; M[p * ld + p] = M[q * ld + q]; M[q * ld + q] = t; }
  for (int64_t j = p + 1; j < q; ++j) {       /* (j, p) <-> (q, j) */
    double t = M[p * ld + j]; M[p * ld + j] = M[j * ld + q]; M[j * ld + q] = t;
  }
  for (int64_t i = q + 1; i < m; ++i) {       /* (i, p) <-> (i, q) */
    double t = M[p * ld + i]; M[p * ld + i] = M[q * ld + i]; M[q * ld + i] = t;
  }
}

/* Eliminate a 1x1 pivot at column k of an m x m lower-stored front (right-looking, rows k+1..m-1). */
static void elim_1x1(double *M, int64_t ld, int64_t m, int64_t k) {
  double d = M[k * ld + k];
  double *col = M + k * ld;
  if (d == 0.0) {           /* zero column (checked by caller): L column is zero */
    for (int64_t i = k + 1; i < m; ++i) col[i] = 0.0;
    return;
  }
  for (int64_t j = k + 1; j < m; ++j) {     /* A22 -= l d l^T with l = col/d, using col = l*d */
    double f = col[j] / d;
    double *cj = M + j * ld;
    for (int64_t i = j; i < m; ++i) cj[i] -= col[i] * f;
  }
  for (int64_t i = k + 1; i < m; ++i) col[i] /= d;
}

/* Eliminate a 2x2 pivot at columns k, k+1. */
static void elim_2x2(double *M, int64_t ld, int64_t m, int64_t k) {
  double a = M[k * ld + k], b = M[k * ld + k + 1], c = M[(k + 1) * ld + k + 1];
  double det = a * c - b * b;
  double *c0 = M + k * ld, *c1 = M + (k + 1) * ld;
  /* W = A21 (m-k-2 x 2), L21 = W E^{-1}, A22 -= W E^{-1} W^T = L21 W^T */
  for (int64_t j = k + 2; j < m; ++j) {
    double w0 = c0[j], w1 = c1[j];
    double l0 = (c * w0 - b * w1) / det, l1 = (a * w1 - b * w0) / det;
    double *cj = M + j * ld;
    for (int64_t i = j; i < m; ++i) cj[i] -= c0[i] * l0 + c1[i] * l1;
  }
  for (int64_t i = k + 2; i < m; ++i) {
    double w0 = c0[i], w1 = c1[i];
    c0[i] = (c * w0 - b * w1) / det;
    c1[i] = (a * w1 - b * w0) / det;
  }
}

/*
 * Unblocked Bunch-Kaufman partial pivoting on columns k0..m-1 of a lower-stored m x m matrix,
 * eliminating every one of them.  perm[] (length m) records the interchanges applied.
 * d[k] / e[k]: diagonal of D and, for a 2x2 block starting at k, its off-diagonal e[k] (e = 0 else).
 */
static void bk_eliminate(double *M, int64_t ld, int64_t m, int64_t k0, int32_t *perm,
                         double *d, double *e, int8_t *piv, orc_inertia *in) {
  int64_t k = k0;
  while (k < m) {
    double akk = fabs(M[k * ld + k]);
    double lam = 0.0; int64_t r = -1;
    for (int64_t i = k + 1; i < m; ++i) {
      double v = fabs(M[k * ld + i]);
      if (v > lam) { lam = v; r = i; }
    }
    int two = 0; int64_t pv = k;
    if (lam == 0.0 && akk == 0.0) {
      pv = k;                                 /* zero column: zero pivot */
    } else if (akk >= BK_ALPHA * lam) {
      pv = k;
    } else {
      double sig = 0.0;
      for (int64_t i = k; i < m; ++i) {
        if (i == r) continue;
        double v = fabs(LO(M, ld, i, r));
        if (v > sig) sig = v;
      }
      if (akk * sig >= BK_ALPHA * lam * lam) pv = k;
      else if (fabs(M[r * ld + r]) >= BK_ALPHA * sig) pv = r;
      else { two = 1; pv = r; }
    }
    if (!two) {
      if (pv != k) { sym_swap(M, ld, m, k, pv); int32_t t = perm[k]; perm[k] = perm[pv]; perm[pv] = t; }
      d[k] = M[k * ld + k]; e[k] = 0.0; piv[k] = 1;
      count_1x1(d[k], in);
      elim_1x1(M, ld, m, k);
      k += 1;
    } else {
      if (pv != k + 1) { sym_swap(M, ld, m, k + 1, pv); int32_t t = perm[k + 1]; perm[k + 1] = perm[pv]; perm[pv] = t; }
      d[k] = M[k * ld + k]; d[k + 1] = M[(k + 1) * ld + k + 1]; e[k] = M[k * ld + k + 1]; e[k + 1] = 0.0;
      piv[k] = 2; piv[k + 1] = 0;
      count_2x2(d[k], e[k], d[k + 1], in);
      elim_2x2(M, ld, m, k);
      k += 2;
    }
  }
}

/*
 * (c1) Dense Bunch-Kaufman LDL^T of the n x n symmetric matrix M (column-major; only the lower
 * triangle is read).  On return M's strict lower triangle holds L (unit diagonal implied; the
 * sub-diagonal entry of each 2x2 block holds that block's off-diagonal, also returned in e),
 * perm maps factor position -> original index, d/e/piv describe D.  Returns the inertia.
 */
void orc_dense_bk(int64_t n, double *M, int32_t *perm, double *d, double *e, int8_t *piv,
                  int64_t *out_neg_zero_pos_n2) {
  orc_inertia in = {0, 0, 0, 0, 0};
  for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
  bk_eliminate(M, n, n, 0, perm, d, e, piv, &in);
  out_neg_zero_pos_n2[0] = in.neg; out_neg_zero_pos_n2[1] = in.zero;
  out_neg_zero_pos_n2[2] = in.pos; out_neg_zero_pos_n2[3] = in.n2x2;
}

/* ------------------------------------------------------------------------------------------ */
/* (c3) sparse multifrontal LDL^T inertia                                                      */
/* ------------------------------------------------------------------------------------------ */

typedef struct {
  int64_t n;
  const int64_t *rp; const int32_t *ci;   /* full symmetric pattern (both triangles) */
} graph_t;

/* Breadth-first levels from root inside the vertex subset marked with tag; returns depth count. */
static int64_t bfs_levels(const graph_t *g, const int32_t *verts, int64_t nv, int32_t root,
                          int32_t *mark, int32_t tag, int32_t *level, int32_t *queue) {
  int64_t head = 0, tail = 0, depth = 0;
  for (int64_t i = 0; i < nv; ++i) level[verts[i]] = -1;
  level[root] = 0; queue[tail++] = root;
  while (head < tail) {
    int32_t v = queue[head++];
    if (level[v] + 1 > depth) depth = level[v] + 1;
    for (int64_t p = g->rp[v]; p < g->rp[v + 1]; ++p) {
      int32_t w = g->ci[p];
      if (mark[w] == tag && level[w] < 0) { level[w] = level[v] + 1; queue[tail++] = w; }
    }
  }
  return tail == nv ? depth : -tail; /* negative: subset not connected from root */
}

typedef struct {
  int64_t nnodes, cap;
  int64_t *first, *count;    /* variables of node t: order[first .. first+count) */
  int64_t *parent;
} ndtree_t;

static int64_t nd_add(ndtree_t *t, int64_t first, int64_t count) {
  if (t->nnodes == t->cap) {
    t->cap = t->cap ? 2 * t->cap : 1024;
    t->first = realloc(t->first, t->cap * sizeof(int64_t));
    t->count = realloc(t->count, t->cap * sizeof(int64_t));
    t->parent = realloc(t->parent, t->cap * sizeof(int64_t));
  }
  t->first[t->nnodes] = first; t->count[t->nnodes] = count; t->parent[t->nnodes] = -1;
  return t->nnodes++;
}

/*
 * Nested dissection by breadth-first level structures: on each connected piece, start from a
 * pseudo-peripheral vertex, take the middle level as the separator, recurse on the two sides.
 * Variables are numbered so every piece comes before its separator; ND tree nodes are created in
 * post-order (children before parents).  The order is written into order[pos .. pos+nv).
 */
static int64_t nd_recurse(const graph_t *g, int32_t *verts, int64_t nv, int64_t pos, int64_t leaf,
                          int32_t *mark, int32_t *tagc, int32_t *level, int32_t *queue,
                          int32_t *order, ndtree_t *tree, int64_t *node_of_child_list,
                          int64_t *nchild) {
  /* returns the ND-tree node id of this subset's top node(s) via node_of_child_list entries */
  if (nv <= leaf) {
    for (int64_t i = 0; i < nv; ++i) order[pos + i] = verts[i];
    int64_t id = nd_add(tree, pos, nv);
    node_of_child_list[(*nchild)++] = id;
    return pos + nv;
  }
  int32_t tag = ++(*tagc);
  for (int64_t i = 0; i < nv; ++i) mark[verts[i]] = tag;
  /* connected component of verts[0] */
  int64_t d = bfs_levels(g, verts, nv, verts[0], mark, tag, level, queue);
  if (d < 0) {
    /* not connected: split into the component reached and the rest, order them one after another
     * (two independent subtrees, no separator) */
    int64_t ncomp = -d;
    int32_t *comp = malloc(ncomp * sizeof(int32_t));
    int32_t *rest = malloc((nv - ncomp) * sizeof(int32_t));
    int64_t a = 0, b = 0;
    for (int64_t i = 0; i < nv; ++i) { if (level[verts[i]] >= 0) comp[a++] = verts[i]; else rest[b++] = verts[i]; }
    pos = nd_recurse(g, comp, a, pos, leaf, mark, tagc, level, queue, order, tree, node_of_child_list, nchild);
    pos = nd_recurse(g, rest, b, pos, leaf, mark, tagc, level, queue, order, tree, node_of_child_list, nchild);
    free(comp); free(rest);
    return pos;
  }
  /* pseudo-peripheral vertex: repeat BFS from a vertex of the last level while depth grows */
  int32_t root = verts[0];
  for (int it = 0; it < 4; ++it) {
    int32_t far = root; int32_t best = -1;
    for (int64_t i = 0; i < nv; ++i) if (level[verts[i]] > best) { best = level[verts[i]]; far = verts[i]; }
    int64_t d2 = bfs_levels(g, verts, nv, far, mark, tag, level, queue);
    if (d2 <= d) { bfs_levels(g, verts, nv, root, mark, tag, level, queue); break; }
    d = d2; root = far;
  }
  if (d < 3) {
    for (int64_t i = 0; i < nv; ++i) order[pos + i] = verts[i];
    int64_t id = nd_add(tree, pos, nv);
    node_of_child_list[(*nchild)++] = id;
    return pos + nv;
  }
  /* middle level as separator, chosen so the two sides are as even as possible */
  int64_t *cnt = calloc(d, sizeof(int64_t));
  for (int64_t i = 0; i < nv; ++i) cnt[level[verts[i]]]++;
  int64_t acc = 0, mid = 1;
  for (int64_t l = 0; l < d; ++l) { acc += cnt[l]; if (2 * acc >= nv) { mid = l; break; } }
  if (mid < 1) mid = 1;
  if (mid > d - 2) mid = d - 2;
  free(cnt);
  int32_t *lo = malloc(nv * sizeof(int32_t)), *hi = malloc(nv * sizeof(int32_t)), *sep = malloc(nv * sizeof(int32_t));
  int64_t nlo = 0, nhi = 0, nsep = 0;
  for (int64_t i = 0; i < nv; ++i) {
    int32_t v = verts[i];
    if (level[v] < mid) lo[nlo++] = v; else if (level[v] > mid) hi[nhi++] = v; else sep[nsep++] = v;
  }
  int64_t mychild[2]; int64_t nmy = 0;
  int64_t *kids = malloc((nv + 2) * sizeof(int64_t)); int64_t nk = 0;
  pos = nd_recurse(g, lo, nlo, pos, leaf, mark, tagc, level, queue, order, tree, kids, &nk);
  pos = nd_recurse(g, hi, nhi, pos, leaf, mark, tagc, level, queue, order, tree, kids, &nk);
  (void)mychild; (void)nmy;
  for (int64_t i = 0; i < nsep; ++i) order[pos + i] = sep[i];
  int64_t id = nd_add(tree, pos, nsep);
  for (int64_t i = 0; i < nk; ++i) tree->parent[kids[i]] = id;
  node_of_child_list[(*nchild)++] = id;
  free(kids); free(lo); free(hi); free(sep);
  return pos + nsep;
}

/* Front record of the oracle's multifrontal elimination. */
typedef struct {
  int64_t m;          /* rows of the contribution block */
  int32_t *rows;      /* its variables (original indices) */
  double *cb;         /* m x m, full symmetric, column-major */
} cbuf_t;

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b; return (x > y) - (x < y);
}

/*
 * Restricted pivoting on the fully-summed columns 0..p-1 of an m x m front held in FULL symmetric
 * column-major storage F (both triangles kept current, plain and slow).  Each accepted pivot is
 * moved to position k (next to eliminate); a column that no acceptable pivot uses stays behind and
 * is passed on (delayed).  Threshold test with u: a 1x1 pivot at j needs |f_jj| >= u * max_i |f_ij|;
 * a 2x2 pivot (j, r) needs every entry of |E^{-1}| [g_j; g_r] <= 1/u with g the column maxima outside
 * the block.  Returns the number of eliminated columns; the caller's inertia is updated.
 */
static void full_swap(double *F, int64_t m, int32_t *rows, int64_t p, int64_t q) {
  if (p == q) return;
  for (int64_t i = 0; i < m; ++i) { double t = F[p * m + i]; F[p * m + i] = F[q * m + i]; F[q * m + i] = t; }
  for (int64_t j = 0; j < m; ++j) { double t = F[j * m + p]; F[j * m + p] = F[j * m + q]; F[j * m + q] = t; }
  int32_t t = rows[p]; rows[p] = rows[q]; rows[q] = t;
}

static double colmax_excl(const double *F, int64_t m, int64_t k, int64_t j, int64_t x1, int64_t x2) {
  double g = 0.0;
  for (int64_t i = k; i < m; ++i) {
    if (i == j || i == x1 || i == x2) continue;
    double v = fabs(F[j * m + i]);
    if (v > g) g = v;
  }
  return g;
}

static void full_elim_1x1(double *F, int64_t m, int64_t k) {
  double d = F[k * m + k];
  if (d == 0.0) return; /* zero column: nothing to subtract */
  for (int64_t j = k + 1; j < m; ++j) {
    double f = F[k * m + j] / d;
    if (f == 0.0) continue;
    for (int64_t i = k + 1; i < m; ++i) F[j * m + i] -= F[k * m + i] * f;
  }
}

static void full_elim_2x2(double *F, int64_t m, int64_t k) {
  double a = F[k * m + k], b = F[k * m + k + 1], c = F[(k + 1) * m + k + 1];
  double det = a * c - b * b;
  for (int64_t j = k + 2; j < m; ++j) {
    double w0 = F[k * m + j], w1 = F[(k + 1) * m + j];
    double l0 = (c * w0 - b * w1) / det, l1 = (a * w1 - b * w0) / det;
    for (int64_t i = k + 2; i < m; ++i) F[j * m + i] -= F[k * m + i] * l0 + F[(k + 1) * m + i] * l1;
  }
}

static int64_t front_eliminate(double *F, int64_t m, int64_t p, int32_t *rows, double u,
                               int is_root, orc_inertia *in) {
  int64_t k = 0;
  while (k < p) {
    int accepted = 0;
    for (int64_t j = k; j < p && !accepted; ++j) {
      double gj = colmax_excl(F, m, k, j, -1, -1);
      double ajj = fabs(F[j * m + j]);
      if (gj == 0.0 || ajj >= u * gj || (is_root && ajj >= BK_ALPHA * gj)) {
        full_swap(F, m, rows, k, j);
        count_1x1(F[k * m + k], in);
        full_elim_1x1(F, m, k);
        k += 1; accepted = 1; break;
      }
      /* best partner r among the remaining fully-summed columns */
      int64_t r = -1; double br = 0.0;
      for (int64_t i = k; i < p; ++i) {
        if (i == j) continue;
        double v = fabs(F[j * m + i]);
        if (v > br) { br = v; r = i; }
      }
      if (r < 0 || br == 0.0) continue;
      double gr = colmax_excl(F, m, k, r, -1, -1);
      if (fabs(F[r * m + r]) >= u * gr && (!is_root || fabs(F[r * m + r]) >= BK_ALPHA * gr)) {
        full_swap(F, m, rows, k, r);
        count_1x1(F[k * m + k], in);
        full_elim_1x1(F, m, k);
        k += 1; accepted = 1; break;
      }
      double a = F[j * m + j], b = F[j * m + r], c = F[r * m + r];
      double det = a * c - b * b;
      if (det == 0.0) continue;
      double gj2 = colmax_excl(F, m, k, j, j, r), gr2 = colmax_excl(F, m, k, r, j, r);
      double t1 = (fabs(c) * gj2 + fabs(b) * gr2) / fabs(det);
      double t2 = (fabs(b) * gj2 + fabs(a) * gr2) / fabs(det);
      if (is_root || (u * t1 <= 1.0 && u * t2 <= 1.0)) {
        full_swap(F, m, rows, k, j);
        if (r == k) r = j;           /* r was moved by the first swap */
        full_swap(F, m, rows, k + 1, r);
        count_2x2(F[k * m + k], F[k * m + k + 1], F[(k + 1) * m + k + 1], in);
        full_elim_2x2(F, m, k);
        k += 2; accepted = 1; break;
      }
    }
    if (!accepted) break;
  }
  return k;
}

/*
 * (c3) Inertia of M = ca*A + cb*B for the symmetric CSR pattern (rp, ci; both triangles stored,
 * A and B on the same pattern).  leaf: largest ND piece left unsplit; u: threshold (0 < u <= 1).
 * out: {neg, zero, pos, delayed, n2x2, nfronts, max_front}.  Returns 0, or -1 on allocation failure.
 */
int orc_sparse_inertia(int64_t n, const int64_t *rp, const int32_t *ci, const double *av,
                       const double *bv, double ca, double cb, int64_t leaf, double u,
                       int64_t *out) {
  graph_t g = {n, rp, ci};
  int32_t *order = malloc(n * sizeof(int32_t)), *mark = calloc(n, sizeof(int32_t));
  int32_t *level = malloc(n * sizeof(int32_t)), *queue = malloc(n * sizeof(int32_t));
  int32_t *verts = malloc(n * sizeof(int32_t));
  int64_t *tops = malloc((n + 2) * sizeof(int64_t)); int64_t ntops = 0;
  if (!order || !mark || !level || !queue || !verts || !tops) return -1;
  for (int64_t i = 0; i < n; ++i) verts[i] = (int32_t)i;
  ndtree_t tree = {0, 0, NULL, NULL, NULL};
  int32_t tagc = 0;
  nd_recurse(&g, verts, n, 0, leaf, mark, &tagc, level, queue, order, &tree, tops, &ntops);
  /* inverse permutation: position of each variable in the elimination order */
  int32_t *posv = malloc(n * sizeof(int32_t));
  for (int64_t i = 0; i < n; ++i) posv[order[i]] = (int32_t)i;
  int64_t nt = tree.nnodes;
  /* children lists */
  int64_t *nch = calloc(nt + 1, sizeof(int64_t));
  for (int64_t t = 0; t < nt; ++t) if (tree.parent[t] >= 0) nch[tree.parent[t] + 1]++;
  for (int64_t t = 0; t < nt; ++t) nch[t + 1] += nch[t];
  int64_t *kid = malloc((nt + 1) * sizeof(int64_t)), *fill = calloc(nt, sizeof(int64_t));
  for (int64_t t = 0; t < nt; ++t) {
    int64_t p = tree.parent[t];
    if (p >= 0) kid[nch[p] + fill[p]++] = t;
  }
  cbuf_t *cbs = calloc(nt, sizeof(cbuf_t));
  orc_inertia in = {0, 0, 0, 0, 0};
  int64_t maxm = 0;
  int32_t *where = malloc(n * sizeof(int32_t));
  for (int64_t i = 0; i < n; ++i) where[i] = -1;
  /* tree nodes are numbered in post-order: children before parents */
  for (int64_t t = 0; t < nt; ++t) {
    int64_t f0 = tree.first[t], nf = tree.count[t];
    /* front variables: own (fully summed), children's contribution rows, own later neighbours */
    int64_t cap = nf;
    for (int64_t c = nch[t]; c < nch[t + 1]; ++c) cap += cbs[kid[c]].m;
    for (int64_t q = f0; q < f0 + nf; ++q) cap += rp[order[q] + 1] - rp[order[q]];
    int32_t *rows = malloc((cap + 1) * sizeof(int32_t));
    int64_t m = 0;
    for (int64_t q = f0; q < f0 + nf; ++q) { rows[m] = order[q]; where[order[q]] = (int32_t)m; m++; }
    /* delayed variables of children join the fully-summed set */
    for (int64_t c = nch[t]; c < nch[t + 1]; ++c) {
      cbuf_t *cbf = &cbs[kid[c]];
      for (int64_t i = 0; i < cbf->m; ++i) {
        int32_t v = cbf->rows[i];
        if (posv[v] < f0 && where[v] < 0) { where[v] = (int32_t)m; rows[m++] = v; }
      }
    }
    int64_t p = m; /* fully summed count */
    int64_t sym_start = m;
    for (int64_t c = nch[t]; c < nch[t + 1]; ++c) {
      cbuf_t *cbf = &cbs[kid[c]];
      for (int64_t i = 0; i < cbf->m; ++i) {
        int32_t v = cbf->rows[i];
        if (where[v] < 0) { where[v] = (int32_t)m; rows[m++] = v; }
      }
    }
    for (int64_t q = f0; q < f0 + nf; ++q) {
      int32_t v = order[q];
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        int32_t w = ci[e];
        if (posv[w] >= f0 + nf && where[w] < 0) { where[w] = (int32_t)m; rows[m++] = w; }
      }
    }
    /* sort the non-fully-summed rows by elimination position (tidy, not needed for correctness) */
    (void)sym_start;
    if (m > maxm) maxm = m;
    double *F = calloc((size_t)m * m, sizeof(double));
    if (!F) return -1;
    /* original entries of columns owned by this node (both triangles of the front) */
    for (int64_t q = f0; q < f0 + nf; ++q) {
      int32_t v = order[q];
      int64_t jv = where[v];
      for (int64_t e = rp[v]; e < rp[v + 1]; ++e) {
        int32_t w = ci[e];
        if (posv[w] < f0) continue;               /* belongs to a descendant's elimination */
        if (posv[w] < posv[v] && posv[w] >= f0 && posv[w] < f0 + nf) continue; /* counted from w */
        int64_t iw = where[w];
        double val = ca * av[e] + cb * bv[e];
        F[jv * m + iw] += val;
        if (iw != jv) F[iw * m + jv] += val;
      }
    }
    /* extend-add children's contribution blocks */
    for (int64_t c = nch[t]; c < nch[t + 1]; ++c) {
      cbuf_t *cbf = &cbs[kid[c]];
      for (int64_t jj = 0; jj < cbf->m; ++jj) {
        int64_t J = where[cbf->rows[jj]];
        for (int64_t ii = 0; ii < cbf->m; ++ii) F[J * m + where[cbf->rows[ii]]] += cbf->cb[jj * cbf->m + ii];
      }
      free(cbf->cb); free(cbf->rows); cbf->cb = NULL; cbf->rows = NULL;
    }
    int is_root = tree.parent[t] < 0;
    int64_t ne = front_eliminate(F, m, p, rows, u, is_root, &in);
    if (is_root && ne < p) {
      /* cannot happen with the root rule above (it accepts the plain Bunch-Kaufman choice) */
      in.delayed += p - ne;
    }
    in.delayed += (is_root ? 0 : p - ne);
    /* contribution block: rows ne..m-1 (delayed first, then the rest) */
    int64_t mc = m - ne;
    if (!is_root && mc > 0) {
      cbs[t].m = mc;
      cbs[t].rows = malloc(mc * sizeof(int32_t));
      cbs[t].cb = malloc((size_t)mc * mc * sizeof(double));
      for (int64_t i = 0; i < mc; ++i) cbs[t].rows[i] = rows[ne + i];
      for (int64_t jj = 0; jj < mc; ++jj)
        for (int64_t ii = 0; ii < mc; ++ii) cbs[t].cb[jj * mc + ii] = F[(ne + jj) * m + ne + ii];
    }
    for (int64_t i = 0; i < m; ++i) where[rows[i]] = -1;
    free(F); free(rows);
  }
  out[0] = in.neg; out[1] = in.zero; out[2] = in.pos; out[3] = in.delayed; out[4] = in.n2x2;
  out[5] = nt; out[6] = maxm;
  free(order); free(mark); free(level); free(queue); free(verts); free(tops); free(posv);
  free(nch); free(kid); free(fill); free(cbs); free(where);
  free(tree.first); free(tree.count); free(tree.parent);
  return 0;
}
