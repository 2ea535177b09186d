/*
 * CPU oracle for the validity test of the linear hexahedron
 * (Johnen, Weill & Remacle, "Robust and efficient validation of the linear
 * hexahedral element", IMR 2017).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, FP64 statement of
 * what the method computes.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load it; the library path never does, and it
 * shares no code, table or constant with the CUDA sources.
 *
 * What it computes, per element (8 nodes, node order of Appendix A):
 *   1. J(xi) = sum_ijk eps_ijk x_i,xi x_j,eta x_k,zeta          (Eq. e:det3d)
 *      from the derivatives of the trilinear shape functions   (Appendix A)
 *   2. c_alpha = J(xi_alpha) at the 27 nodes of the order-2 hexahedron,
 *      ordered as in Fig. f:ordercoeff (Sec. 3.2)
 *   3. b = T c with the matrix of Table t:Tb                    (Sec. 3.2)
 *   4. the decision of Sec. 6: 20 sampled values (corners + edge midpoints)
 *      non-positive -> invalid; all 27 coefficients positive -> valid; else
 *      subdivide (quadratic de Casteljau split at 1/2 along xi, eta, zeta) and
 *      test each sub-box: a non-positive corner coefficient -> invalid, all 27
 *      positive -> that box is certified, otherwise refine it further.
 *
 * The refinement is evaluated level by level (breadth first) with a depth cap
 * D, which gives an order-independent verdict and decision depth:
 *   INVALID@d   d = the shallowest level holding a non-positive corner value
 *   VALID@d     d = the level of the deepest certified box
 *   UNDECIDED@D the cap was reached with uncertified boxes and no invalid one.
 *
 * Every sign decision is certified: each computed value carries a rigorous
 * forward-error bound (a priori bound of the "absolute value" expression
 * tree), and a value whose sign the bound cannot settle marks the element
 * AMBIGUOUS; the Python side then recomputes that element in exact rational
 * arithmetic.  The flags are therefore those of exact arithmetic on the FP64
 * input values.  bmin/bmax are the min/max of the 27 depth-0 coefficients.
 *
 * Flag byte: bits 0-2 verdict (1 valid, 2 invalid, 3 undecided, 4 non-finite
 * input), bits 3-6 decision depth, bit 7 "needed the exact tier" (diagnostic).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define V_VALID 1
#define V_INVALID 2
#define V_UNDECIDED 3
#define V_NONFINITE 4
#define F_AMBIGUOUS 0x80 /* internal return: exact tier required */

/* Appendix A: reference coordinates of nodes 1..8. */
static const int REF_NODE[8][3] = {
    {0, 0, 0}, {1, 0, 0}, {1, 1, 0}, {0, 1, 0},
    {0, 0, 1}, {1, 0, 1}, {1, 1, 1}, {0, 1, 1}};

/* Fig. f:ordercoeff: the 27 nodes of the order-2 hexahedron, coordinates x2.
 * 1-8 corners, 9-20 edge midpoints (edges 12,23,34,41,15,26,37,48,56,67,78,85),
 * 21-26 face centres (faces zeta=0, eta=0, xi=1, eta=1, xi=0, zeta=1), 27 centre. */
static const int LAT2[27][3] = {
    {0, 0, 0}, {2, 0, 0}, {2, 2, 0}, {0, 2, 0}, {0, 0, 2}, {2, 0, 2}, {2, 2, 2}, {0, 2, 2},
    {1, 0, 0}, {2, 1, 0}, {1, 2, 0}, {0, 1, 0}, {0, 0, 1}, {2, 0, 1}, {2, 2, 1}, {0, 2, 1},
    {1, 0, 2}, {2, 1, 2}, {1, 2, 2}, {0, 1, 2},
    {1, 1, 0}, {1, 0, 1}, {2, 1, 1}, {1, 2, 1}, {0, 1, 1}, {1, 1, 2},
    {1, 1, 1}};

/* Table t:Tb, built block by block as the table prints it (1-based node ids). */
static const int EDGE_END[12][2] = {{1, 2}, {2, 3}, {3, 4}, {1, 4}, {1, 5}, {2, 6},
                                    {3, 7}, {4, 8}, {5, 6}, {6, 7}, {7, 8}, {5, 8}};
static const int FACE_CORNER[6][4] = {{1, 2, 3, 4}, {1, 2, 5, 6}, {2, 3, 6, 7},
                                      {3, 4, 7, 8}, {1, 4, 5, 8}, {5, 6, 7, 8}};
static const int FACE_EDGE[6][4] = {{9, 10, 11, 12}, {9, 13, 14, 17}, {10, 14, 15, 18},
                                    {11, 15, 16, 19}, {12, 13, 16, 20}, {17, 18, 19, 20}};

static double T[27][27];
static int T_ready = 0;

static void build_T(void) {
  if (T_ready) return;
  memset(T, 0, sizeof(T));
  for (int r = 0; r < 8; ++r) T[r][r] = 1.0;                /* identity block */
  for (int e = 0; e < 12; ++e) {                            /* edge rows */
    int r = 8 + e;
    T[r][EDGE_END[e][0] - 1] = -0.5;
    T[r][EDGE_END[e][1] - 1] = -0.5;
    T[r][r] = 2.0;
  }
  for (int f = 0; f < 6; ++f) {                             /* face rows */
    int r = 20 + f;
    for (int q = 0; q < 4; ++q) {
      T[r][FACE_CORNER[f][q] - 1] = 0.25;
      T[r][FACE_EDGE[f][q] - 1] = -1.0;
    }
    T[r][r] = 4.0;
  }
  for (int a = 0; a < 8; ++a) T[26][a] = -0.125;            /* centre row */
  for (int a = 8; a < 20; ++a) T[26][a] = 0.5;
  for (int a = 20; a < 26; ++a) T[26][a] = -2.0;
  T[26][26] = 8.0;
  T_ready = 1;
}

/* Unit roundoff u of binary64 and the bound constants.  Standard forward
 * error analysis (Higham, "Accuracy and Stability of Numerical Algorithms",
 * ch. 3): a value built from sums and products in which every term passes
 * through at most k roundings lies within gamma_k = k u / (1 - k u) times the
 * same expression evaluated on absolute values of its exact value.  In
 * jac_det the shape-function derivatives at the lattice points are 0, +-1/4,
 * +-1/2 or +-1, so the products X * d are exact; a Jacobian entry then passes
 * through 7 roundings (8 terms summed), a determinant term through 2 more (a
 * product of three entries) and the signed sum of the 6 terms through 5
 * more: <= 14 per J sample, bounded by 15 here.  A Bezier coefficient adds
 * the dyadic weights of its row of Table t:Tb (exact products) and <= 26
 * additions: with |c - c_exact| <= gamma_15 M, |b - b_exact| <= gamma_41
 * sum |T| M.  One subdivision level forms each child coefficient by three
 * de Casteljau passes of two averages each (the halvings are exact): <= 6
 * roundings of a convex combination, so gamma_6 max |b| more.  K_C, K_B and
 * K_SUB are 2 gamma_15, 2 gamma_41 and gamma_6 rounded up (the factor covers
 * the 1 / (1 - k u) denominators); E_FLOOR covers the absolute errors of
 * gradual underflow. */
#define U64 (1.1102230246251565e-16) /* 2^-53 */
#define K_C (32.0 * U64)             /* >= 2 * gamma_15 inflation */
#define K_B (128.0 * U64)            /* >= 2 * gamma_41 inflation */
#define K_SUB (8.0 * U64)            /* >= gamma_6 with inflation */
#define E_FLOOR (1e-300)             /* absorbs gradual-underflow errors */

/* Derivative of shape function k (Appendix A) w.r.t. reference axis j at xi. */
static double dshape(int k, int j, const double xi[3]) {
  double v = 1.0;
  for (int d = 0; d < 3; ++d) {
    double l = REF_NODE[k][d] ? xi[d] : 1.0 - xi[d];
    double dl = REF_NODE[k][d] ? 1.0 : -1.0;
    v *= (d == j) ? dl : l;
  }
  return v;
}

/* Eq. e:det3d at xi.  *mag receives the same expression evaluated on absolute
 * values (every subtraction replaced by an addition), which bounds the
 * rounding error: |J_computed - J| <= gamma_15 * mag. */
static double jac_det(const double X[8][3], const double xi[3], double* mag) {
  double Jm[3][3], A[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0, sa = 0.0;
      for (int k = 0; k < 8; ++k) {
        double d = dshape(k, j, xi);
        s += X[k][i] * d;
        sa += fabs(X[k][i]) * fabs(d);
      }
      Jm[i][j] = s; /* x_i,xi_j */
      A[i][j] = sa;
    }
  /* sum over permutations (i,j,k) of eps_ijk x_i,xi x_j,eta x_k,zeta */
  static const int P[6][3] = {{0, 1, 2}, {1, 2, 0}, {2, 0, 1}, {0, 2, 1}, {2, 1, 0}, {1, 0, 2}};
  static const double S[6] = {1, 1, 1, -1, -1, -1};
  double J = 0.0, M = 0.0;
  for (int p = 0; p < 6; ++p) {
    J += S[p] * Jm[P[p][0]][0] * Jm[P[p][1]][1] * Jm[P[p][2]][2];
    M += A[P[p][0]][0] * A[P[p][1]][1] * A[P[p][2]][2];
  }
  *mag = M;
  return J;
}

/* Public helper: J at an arbitrary reference point. */
double oracle_jacobian(const double* X24, double xi, double eta, double zeta) {
  double X[8][3], p[3] = {xi, eta, zeta}, m;
  memcpy(X, X24, sizeof(X));
  return jac_det(X, p, &m);
}

/* Samples c (27), coefficients b = T c (27) and their error bounds. */
static void coefficients(const double X[8][3], double c[27], double ec[27], double b[27],
                         double eb[27]) {
  build_T();
  double M[27];
  for (int a = 0; a < 27; ++a) {
    double xi[3] = {0.5 * LAT2[a][0], 0.5 * LAT2[a][1], 0.5 * LAT2[a][2]};
    c[a] = jac_det(X, xi, &M[a]);
    ec[a] = K_C * M[a] + E_FLOOR;
  }
  for (int r = 0; r < 27; ++r) {
    double s = 0.0, sm = 0.0;
    for (int a = 0; a < 27; ++a) {
      s += T[r][a] * c[a];
      sm += fabs(T[r][a]) * M[a];
    }
    b[r] = s;
    eb[r] = K_B * sm + E_FLOOR;
  }
}

/* Public helper for tests: samples and coefficients of one element. */
void oracle_coefficients(const double* X24, double* c27, double* b27) {
  double X[8][3], ec[27], eb[27];
  memcpy(X, X24, sizeof(X));
  coefficients(X, c27, ec, b27, eb);
}

/* Public helper for tests: coefficients and their certified error bounds. */
void oracle_coefficient_bounds(const double* X24, double* b27, double* eb27) {
  double X[8][3], c[27], ec[27];
  memcpy(X, X24, sizeof(X));
  coefficients(X, c, ec, b27, eb27);
}

/* Tensor index (i,j,k) in {0,1,2}^3 of coefficient alpha is LAT2[alpha]. */
static int alpha_of[3][3][3];
static int alpha_ready = 0;
static void build_alpha(void) {
  if (alpha_ready) return;
  for (int a = 0; a < 27; ++a) alpha_of[LAT2[a][0]][LAT2[a][1]][LAT2[a][2]] = a;
  alpha_ready = 1;
}

/* Quadratic de Casteljau split at 1/2 along xi, eta, zeta: the 8 children of
 * a box, child o = sx + 2 sy + 4 sz covering [sx/2,(sx+1)/2] x ... of it.
 * On a line (p0,p1,p2): left = (p0, (p0+p1)/2, (p0+2p1+p2)/4),
 * right = ((p0+2p1+p2)/4, (p1+p2)/2, p2). */
static void subdivide(const double b[27], double child[8][27]) {
  build_alpha();
  double G[5][5][5]; /* after the three passes: 5 points per axis */
  double A0[3][3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) A0[i][j][k] = b[alpha_of[i][j][k]];
  double A1[5][3][3], A2[5][5][3];
  for (int j = 0; j < 3; ++j)
    for (int k = 0; k < 3; ++k) { /* along xi */
      double p0 = A0[0][j][k], p1 = A0[1][j][k], p2 = A0[2][j][k];
      double l1 = (p0 + p1) * 0.5, r1 = (p1 + p2) * 0.5;
      A1[0][j][k] = p0; A1[1][j][k] = l1; A1[2][j][k] = (l1 + r1) * 0.5;
      A1[3][j][k] = r1; A1[4][j][k] = p2;
    }
  for (int i = 0; i < 5; ++i)
    for (int k = 0; k < 3; ++k) { /* along eta */
      double p0 = A1[i][0][k], p1 = A1[i][1][k], p2 = A1[i][2][k];
      double l1 = (p0 + p1) * 0.5, r1 = (p1 + p2) * 0.5;
      A2[i][0][k] = p0; A2[i][1][k] = l1; A2[i][2][k] = (l1 + r1) * 0.5;
      A2[i][3][k] = r1; A2[i][4][k] = p2;
    }
  for (int i = 0; i < 5; ++i)
    for (int j = 0; j < 5; ++j) { /* along zeta */
      double p0 = A2[i][j][0], p1 = A2[i][j][1], p2 = A2[i][j][2];
      double l1 = (p0 + p1) * 0.5, r1 = (p1 + p2) * 0.5;
      G[i][j][0] = p0; G[i][j][1] = l1; G[i][j][2] = (l1 + r1) * 0.5;
      G[i][j][3] = r1; G[i][j][4] = p2;
    }
  for (int o = 0; o < 8; ++o) {
    int sx = o & 1, sy = (o >> 1) & 1, sz = (o >> 2) & 1;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
          child[o][alpha_of[i][j][k]] = G[2 * sx + i][2 * sy + j][2 * sz + k];
  }
}

/* Public helper for tests. */
void oracle_subdivide(const double* b27, double* children216) {
  double ch[8][27];
  subdivide(b27, ch);
  memcpy(children216, ch, sizeof(ch));
}

/* Error bound of the children of a box whose 27 computed coefficients b
 * carry the uniform bound e_parent: the children are convex combinations
 * formed with at most 6 roundings, each at most u times the largest |b|. */
static double child_bound(double e_parent, const double b[27]) {
  double bm = 0.0;
  for (int a = 0; a < 27; ++a)
    if (fabs(b[a]) > bm) bm = fabs(b[a]);
  return e_parent + K_SUB * bm + E_FLOOR;
}

double oracle_child_bound(double e_parent, const double* b27) {
  return child_bound(e_parent, b27);
}

/* Certified sign classes of a computed value v with error bound e. */
#define S_NONPOS 0 /* exact value certainly <= 0 */
#define S_POS 1    /* exact value certainly > 0 */
#define S_AMBIG 2

static int sign_class(double v, double e) {
  if (v <= -e) return S_NONPOS;
  if (v > e) return S_POS;
  return S_AMBIG;
}

typedef struct {
  double b[27];
  double e; /* uniform error bound of the 27 values */
} box_t;

/* Decide one element.  Returns the flag byte, or F_AMBIGUOUS when some sign
 * decision on which the verdict depends could not be certified. */
static int decide(const double X[8][3], int max_depth, double* bmin, double* bmax) {
  for (int k = 0; k < 8; ++k)
    for (int i = 0; i < 3; ++i)
      if (!isfinite(X[k][i])) {
        *bmin = NAN;
        *bmax = NAN;
        return V_NONFINITE;
      }
  double c[27], ec[27], b[27], eb[27];
  coefficients(X, c, ec, b, eb);
  double lo = b[0], hi = b[0];
  for (int a = 1; a < 27; ++a) {
    if (b[a] < lo) lo = b[a];
    if (b[a] > hi) hi = b[a];
  }
  *bmin = lo;
  *bmax = hi;

  /* Level 0, Sec. 6 Step 2: the 20 samples (8 corners and 12 edge midpoints). */
  int any_nonpos = 0, any_ambig = 0;
  for (int a = 0; a < 20; ++a) {
    int s = sign_class(c[a], ec[a]);
    any_nonpos |= (s == S_NONPOS);
    any_ambig |= (s == S_AMBIG);
  }
  if (any_nonpos) return V_INVALID | (0 << 3);
  if (any_ambig) return F_AMBIGUOUS;
  /* Step 4: all 27 coefficients positive -> valid. */
  int certified = 1;
  double e0 = 0.0;
  for (int a = 0; a < 27; ++a) {
    int s = sign_class(b[a], eb[a]);
    if (s == S_AMBIG) return F_AMBIGUOUS;
    if (s == S_NONPOS) certified = 0;
    if (eb[a] > e0) e0 = eb[a];
  }
  if (certified) return V_VALID | (0 << 3);
  if (max_depth == 0) return V_UNDECIDED | (0 << 3);

  /* Step 5: refinement, breadth first. */
  size_t cap = 64, n = 1;
  box_t* cur = (box_t*)malloc(cap * sizeof(box_t));
  memcpy(cur[0].b, b, sizeof(b));
  cur[0].e = e0;
  int result = F_AMBIGUOUS;
  for (int level = 1; level <= max_depth; ++level) {
    size_t ncap = 8 * n, m = 0;
    box_t* kids = (box_t*)malloc(ncap * sizeof(box_t));
    for (size_t q = 0; q < n; ++q) {
      double ch[8][27];
      subdivide(cur[q].b, ch);
      double echild = child_bound(cur[q].e, cur[q].b);
      for (int o = 0; o < 8; ++o) {
        memcpy(kids[m].b, ch[o], sizeof(ch[o]));
        kids[m].e = echild;
        ++m;
      }
    }
    free(cur);
    /* corners of every box of this level (Sec. 6, subdivision Step 3) */
    any_nonpos = 0;
    any_ambig = 0;
    for (size_t q = 0; q < m; ++q)
      for (int a = 0; a < 8; ++a) {
        int s = sign_class(kids[q].b[a], kids[q].e);
        any_nonpos |= (s == S_NONPOS);
        any_ambig |= (s == S_AMBIG);
      }
    if (any_nonpos) { result = V_INVALID | (level << 3); free(kids); goto done; }
    if (any_ambig) { result = F_AMBIGUOUS; free(kids); goto done; }
    /* certification of every box (subdivision Step 4) */
    size_t keep = 0;
    for (size_t q = 0; q < m; ++q) {
      int cert = 1;
      for (int a = 8; a < 27; ++a) {
        int s = sign_class(kids[q].b[a], kids[q].e);
        if (s == S_AMBIG) { result = F_AMBIGUOUS; free(kids); goto done; }
        if (s == S_NONPOS) cert = 0;
      }
      if (!cert) kids[keep++] = kids[q];
    }
    if (keep == 0) { result = V_VALID | (level << 3); free(kids); goto done; }
    if (level == max_depth) { result = V_UNDECIDED | (level << 3); free(kids); goto done; }
    cur = kids;
    n = keep;
    cap = ncap;
  }
done:
  (void)cap;
  return result;
}

static void gather_soa(const double* corners, int64_t n, int64_t e, double X[8][3]) {
  for (int k = 0; k < 8; ++k)
    for (int i = 0; i < 3; ++i) X[k][i] = corners[((int64_t)(k * 3 + i)) * n + e];
}

/* corners: SoA planes [8][3][n] (node-major, then x/y/z).  flags gets the
 * flag byte, or 0x80 for elements that need the exact tier. */
int oracle_check_soa(int64_t n, const double* corners, int max_depth, int threads,
                     uint8_t* flags, double* bmin, double* bmax) {
  if (n < 0 || max_depth < 0 || max_depth > 15) return -1;
  build_T();
  build_alpha();
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
  for (int64_t e = 0; e < n; ++e) {
    double X[8][3], lo, hi;
    gather_soa(corners, n, e, X);
    flags[e] = (uint8_t)decide(X, max_depth, &lo, &hi);
    bmin[e] = lo;
    bmax[e] = hi;
  }
  return 0;
}

/* nodes: [n_nodes][3]; conn: [n_hex][8] 0-based node ids in Appendix A order.
 * Returns -2 if a connectivity entry is out of range. */
int oracle_check_indexed(int64_t n_nodes, const double* nodes, int64_t n_hex,
                         const int32_t* conn, int max_depth, int threads, uint8_t* flags,
                         double* bmin, double* bmax) {
  if (n_hex < 0 || n_nodes < 0 || max_depth < 0 || max_depth > 15) return -1;
  for (int64_t e = 0; e < n_hex * 8; ++e)
    if (conn[e] < 0 || conn[e] >= n_nodes) return -2;
  build_T();
  build_alpha();
#ifdef _OPENMP
  if (threads > 0) omp_set_num_threads(threads);
#pragma omp parallel for schedule(dynamic, 256)
#endif
  for (int64_t e = 0; e < n_hex; ++e) {
    double X[8][3], lo, hi;
    for (int k = 0; k < 8; ++k)
      for (int i = 0; i < 3; ++i) X[k][i] = nodes[(int64_t)conn[e * 8 + k] * 3 + i];
    flags[e] = (uint8_t)decide(X, max_depth, &lo, &hi);
    bmin[e] = lo;
    bmax[e] = hi;
  }
  return 0;
}

int oracle_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
