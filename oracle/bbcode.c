/*
 * bbcode.c -- CPU ORACLE (test infrastructure only): bivariate-bicycle code
 * construction and GF(2) linear algebra, written out with dense 0/1 matrices.
 *
 * BB code (appendix "Single shot syndrome noise"): H_X = [A | B] with
 * x = S_l (x) I_m, y = I_l (x) S_m, S the cyclic shift; a monomial x^a y^b is
 * the position m*a + b of a length-lm vector.  The worked example of that
 * appendix (first columns b_1 = y^5 + y^10 + x^9 of A = x^3 + y^2 + y^7) fixes
 * the shift direction as S[i][(i+1) mod l] = 1.  H_Z = [B^T | A^T] is the
 * reading for which H_X H_Z^T = AB + BA = 0.
 */
#include "qdo.h"
#include <stdlib.h>
#include <string.h>

/* Dense l x l cyclic shift raised to the power a: S^a[i][(i+a) mod l] = 1. */
static void shift_pow(int l, int a, uint8_t* S) {
  memset(S, 0, (size_t)l * l);
  for (int i = 0; i < l; ++i) S[i * l + (((i + a) % l) + l) % l] = 1;
}

/* Kronecker product P (x) Q of an l x l and an m x m matrix. */
static void kron(int l, const uint8_t* P, int m, const uint8_t* Q, uint8_t* out) {
  int w = l * m;
  for (int i1 = 0; i1 < l; ++i1)
    for (int j1 = 0; j1 < l; ++j1)
      for (int i2 = 0; i2 < m; ++i2)
        for (int j2 = 0; j2 < m; ++j2)
          out[(size_t)(i1 * m + i2) * w + (j1 * m + j2)] = P[i1 * l + j1] & Q[i2 * m + j2];
}

/* One monomial x^a y^b as a dense lm x lm matrix. */
static void monomial(int l, int m, int a, int b, uint8_t* out) {
  uint8_t* Sx = malloc((size_t)l * l);
  uint8_t* Sy = malloc((size_t)m * m);
  shift_pow(l, a, Sx);
  shift_pow(m, b, Sy);
  kron(l, Sx, m, Sy, out);
  free(Sx);
  free(Sy);
}

/* Dense A (or B) = sum of three monomials, over GF(2). */
static void poly3(int l, int m, const int* ex, const int* ey, uint8_t* out) {
  int w = l * m;
  uint8_t* t = malloc((size_t)w * w);
  memset(out, 0, (size_t)w * w);
  for (int k = 0; k < 3; ++k) {
    monomial(l, m, ex[k], ey[k], t);
    for (size_t q = 0; q < (size_t)w * w; ++q) out[q] ^= t[q];
  }
  free(t);
}

int qdo_code_matrices(const qdo_code* c, uint8_t* HX, uint8_t* HZ) {
  int w = c->l * c->m, n = 2 * w;
  uint8_t* A = malloc((size_t)w * w);
  uint8_t* B = malloc((size_t)w * w);
  poly3(c->l, c->m, c->ax, c->ay, A);
  poly3(c->l, c->m, c->bx, c->by, B);
  for (int i = 0; i < w; ++i)
    for (int j = 0; j < w; ++j) {
      HX[(size_t)i * n + j] = A[(size_t)i * w + j];
      HX[(size_t)i * n + w + j] = B[(size_t)i * w + j];
      HZ[(size_t)i * n + j] = B[(size_t)j * w + i];     /* B^T */
      HZ[(size_t)i * n + w + j] = A[(size_t)j * w + i]; /* A^T */
    }
  free(A);
  free(B);
  return 0;
}

/* Rank over GF(2) by Gaussian elimination on a copy. */
int qdo_gf2_rank(const uint8_t* M, int rows, int cols) {
  uint8_t* a = malloc((size_t)rows * cols);
  memcpy(a, M, (size_t)rows * cols);
  int rank = 0;
  for (int c = 0; c < cols && rank < rows; ++c) {
    int piv = -1;
    for (int r = rank; r < rows; ++r)
      if (a[(size_t)r * cols + c]) { piv = r; break; }
    if (piv < 0) continue;
    if (piv != rank)
      for (int k = 0; k < cols; ++k) {
        uint8_t t = a[(size_t)piv * cols + k];
        a[(size_t)piv * cols + k] = a[(size_t)rank * cols + k];
        a[(size_t)rank * cols + k] = t;
      }
    for (int r = 0; r < rows; ++r)
      if (r != rank && a[(size_t)r * cols + c])
        for (int k = 0; k < cols; ++k) a[(size_t)r * cols + k] ^= a[(size_t)rank * cols + k];
    ++rank;
  }
  free(a);
  return rank;
}

/*
 * Logical operators of one type: vectors v with Hk v = 0 (they commute with
 * every check of Hk) that are independent modulo the row span of Hr.  A
 * kernel basis of Hk comes from its reduced row echelon form (Hk is reduced in
 * place); kernel vectors are then added greedily whenever they raise the rank
 * of [Hr; chosen].  Both matrices are w x n.  Returns K.
 */
static int logical_basis(uint8_t* HX, const uint8_t* HZ, int w, int n, uint8_t* LZ, int max_k) {
  /* RREF of the kernel matrix */
  int* pivcol = malloc(sizeof(int) * w);
  int rank = 0;
  for (int col = 0; col < n && rank < w; ++col) {
    int piv = -1;
    for (int r = rank; r < w; ++r)
      if (HX[(size_t)r * n + col]) { piv = r; break; }
    if (piv < 0) continue;
    if (piv != rank)
      for (int k = 0; k < n; ++k) {
        uint8_t t = HX[(size_t)piv * n + k];
        HX[(size_t)piv * n + k] = HX[(size_t)rank * n + k];
        HX[(size_t)rank * n + k] = t;
      }
    for (int r = 0; r < w; ++r)
      if (r != rank && HX[(size_t)r * n + col])
        for (int k = 0; k < n; ++k) HX[(size_t)r * n + k] ^= HX[(size_t)rank * n + k];
    pivcol[rank++] = col;
  }
  uint8_t* isp = calloc(n, 1);
  for (int r = 0; r < rank; ++r) isp[pivcol[r]] = 1;
  /* stack = rows of the row-span matrix followed by chosen logicals */
  int cap = w + max_k + 1;
  uint8_t* stack = malloc((size_t)cap * n);
  memcpy(stack, HZ, (size_t)w * n);
  int base_rank = qdo_gf2_rank(stack, w, n);
  int K = 0;
  uint8_t* v = malloc(n);
  for (int f = 0; f < n && K < max_k; ++f) {
    if (isp[f]) continue;
    /* kernel vector with free variable f set: pivot variables follow from RREF */
    memset(v, 0, n);
    v[f] = 1;
    for (int r = 0; r < rank; ++r)
      if (HX[(size_t)r * n + f]) v[pivcol[r]] = 1;
    memcpy(stack + (size_t)(w + K) * n, v, n);
    int rk = qdo_gf2_rank(stack, w + K + 1, n);
    if (rk > base_rank + K) {
      memcpy(LZ + (size_t)K * n, v, n);
      ++K;
    }
  }
  free(v);
  free(stack);
  free(isp);
  free(pivcol);
  return K;
}

/* Logical Z operators of the Z-basis memory: kernel of H_X modulo the row
 * span of H_Z.  Returns K. */
int qdo_logical_z(const qdo_code* c, uint8_t* LZ, int max_k) {
  int w = c->l * c->m, n = 2 * w;
  uint8_t* HX = malloc((size_t)w * n);
  uint8_t* HZ = malloc((size_t)w * n);
  qdo_code_matrices(c, HX, HZ);
  int K = logical_basis(HX, HZ, w, n, LZ, max_k);
  free(HX);
  free(HZ);
  return K;
}

/* Logical operators seen by errors decoded with H_X (appendices A and B):
 * kernel of H_Z modulo the row span of H_X.  Returns K. */
int qdo_logical_x(const qdo_code* c, uint8_t* LX, int max_k) {
  int w = c->l * c->m, n = 2 * w;
  uint8_t* HX = malloc((size_t)w * n);
  uint8_t* HZ = malloc((size_t)w * n);
  qdo_code_matrices(c, HX, HZ);
  int K = logical_basis(HZ, HX, w, n, LX, max_k);
  free(HX);
  free(HZ);
  return K;
}
