/*
 * CPU oracle for the LCS table fill and traceback — TEST INFRASTRUCTURE ONLY.
 *
 * Only the tests, the smoke check and the CPU-baseline leg of the benchmark may load this file's library. The
 * product path (the CUDA library) shares no code with it and never calls it.
 *
 * It is the paper's method written out literally and slowly (Dash & Nayak, "Parallel Algorithm for Longest Common
 * Subsequence in a String"):
 *   - LCS-length (§I.C): the table c[0..m, 0..n] is filled in row-major order; c = 0 on the borders; on a match
 *     x_i = y_j, c[i,j] = c[i-1,j-1] + 1 and b[i,j] = DIAG; otherwise, if c[i-1,j] >= c[i,j-1], c[i,j] = c[i-1,j]
 *     and b[i,j] = UP, else c[i,j] = c[i,j-1] and b[i,j] = LEFT. c[m,n] is the LCS length.
 *   - Print-LCS (§I.D): start at b[m,n] and follow the arrows; every DIAG cell contributes x_i; the symbols come
 *     out in reverse order. The paper's listing is garbled in its UP branch and omits the LEFT branch; this file
 *     follows the textbook reading the paper cites: DIAG -> (i-1, j-1) and emit x_i, UP -> (i-1, j),
 *     LEFT -> (i, j-1), stop when i = 0 or j = 0.
 * X has length m and indexes the rows, Y has length n and indexes the columns (the theorem of §I.A uses x_m, y_n).
 * Symbols are bytes compared for equality.
 *
 * Storage choices that do not change any value: c is kept as two rolling rows of uint32 (the full table would be
 * 17 GB at m = n = 65536), b is stored at 2 bits per cell, and Print-LCS is an explicit loop instead of recursion
 * (a recursion depth of m + n would overflow the stack).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { ORACLE_DIAG = 1, ORACLE_UP = 2, ORACLE_LEFT = 3 };
enum { ORACLE_OK = 0, ORACLE_ERR_NOMEM = -1, ORACLE_ERR_CAPACITY = -2, ORACLE_ERR_INVALID = -3 };

/* LCS-length (§I.C), length only: row-major fill of c with the recurrence above; returns c[m,n]. */
uint64_t oracle_lcs_length(const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n) {
  if (m == 0 || n == 0) return 0;
  uint32_t* prev = (uint32_t*)calloc(n + 1, sizeof(uint32_t)); /* c[i-1][0..n], starts as row 0 = 0 */
  uint32_t* cur = (uint32_t*)calloc(n + 1, sizeof(uint32_t));  /* c[i][0..n] */
  if (!prev || !cur) { free(prev); free(cur); return UINT64_MAX; }
  for (uint64_t i = 1; i <= m; ++i) {
    cur[0] = 0; /* c[i,0] = 0 */
    for (uint64_t j = 1; j <= n; ++j) {
      if (x[i - 1] == y[j - 1]) {
        cur[j] = prev[j - 1] + 1;
      } else if (prev[j] >= cur[j - 1]) {
        cur[j] = prev[j];
      } else {
        cur[j] = cur[j - 1];
      }
    }
    uint32_t* t = prev; prev = cur; cur = t;
  }
  uint64_t len = prev[n];
  free(prev); free(cur);
  return len;
}

static inline void b_set(uint8_t* b, uint64_t cell, unsigned v) {
  b[cell >> 2] |= (uint8_t)(v << ((cell & 3) * 2));
}
static inline unsigned b_get(const uint8_t* b, uint64_t cell) {
  return (b[cell >> 2] >> ((cell & 3) * 2)) & 3u;
}

/* LCS-length (§I.C) with the b table, then Print-LCS (§I.D). Writes the LCS into out[0..len) and its length into
 * *out_len. Returns ORACLE_ERR_CAPACITY (with *out_len = the length) when out_cap < len. */
int oracle_lcs_traceback(const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint8_t* out,
                         uint64_t out_cap, uint64_t* out_len) {
  if (!out_len) return ORACLE_ERR_INVALID;
  *out_len = 0;
  if (m == 0 || n == 0) return ORACLE_OK;
  uint64_t cells = m * n;
  if (cells / m != n) return ORACLE_ERR_INVALID;
  uint8_t* b = (uint8_t*)calloc((cells + 3) / 4, 1); /* b[1..m, 1..n], cell (i,j) at (i-1)*n + (j-1) */
  uint32_t* prev = (uint32_t*)calloc(n + 1, sizeof(uint32_t));
  uint32_t* cur = (uint32_t*)calloc(n + 1, sizeof(uint32_t));
  uint8_t* rev = (uint8_t*)malloc(m < n ? m : n);
  if (!b || !prev || !cur || !rev) { free(b); free(prev); free(cur); free(rev); return ORACLE_ERR_NOMEM; }
  for (uint64_t i = 1; i <= m; ++i) {
    cur[0] = 0;
    for (uint64_t j = 1; j <= n; ++j) {
      uint64_t cell = (i - 1) * n + (j - 1);
      if (x[i - 1] == y[j - 1]) {
        cur[j] = prev[j - 1] + 1;
        b_set(b, cell, ORACLE_DIAG);
      } else if (prev[j] >= cur[j - 1]) {
        cur[j] = prev[j];
        b_set(b, cell, ORACLE_UP);
      } else {
        cur[j] = cur[j - 1];
        b_set(b, cell, ORACLE_LEFT);
      }
    }
    uint32_t* t = prev; prev = cur; cur = t;
  }
  uint64_t len = prev[n];
  /* Print-LCS (§I.D) from b[m,n]: symbols are met in reverse order. */
  uint64_t i = m, j = n, k = 0;
  while (i > 0 && j > 0) {
    unsigned d = b_get(b, (i - 1) * n + (j - 1));
    if (d == ORACLE_DIAG) {
      rev[k++] = x[i - 1];
      --i; --j;
    } else if (d == ORACLE_UP) {
      --i;
    } else {
      --j;
    }
  }
  free(b); free(prev); free(cur);
  *out_len = len;
  if (k != len) { free(rev); return ORACLE_ERR_INVALID; } /* cannot happen: every DIAG step adds exactly 1 */
  if (out_cap < len) { free(rev); return ORACLE_ERR_CAPACITY; }
  for (uint64_t t = 0; t < len; ++t) out[t] = rev[len - 1 - t];
  free(rev);
  return ORACLE_OK;
}

/* The full tables returned by LCS-length (§I.C): c[(m+1)*(n+1)] row-major (row i over X) and b[m*n] row-major,
 * b holding ORACLE_DIAG / ORACLE_UP / ORACLE_LEFT. For small inputs (tests and table export checks). */
int oracle_lcs_tables(const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint32_t* c, uint8_t* b) {
  uint64_t w = n + 1;
  for (uint64_t j = 0; j <= n; ++j) c[j] = 0;
  for (uint64_t i = 1; i <= m; ++i) {
    c[i * w] = 0;
    for (uint64_t j = 1; j <= n; ++j) {
      uint32_t diag = c[(i - 1) * w + (j - 1)], up = c[(i - 1) * w + j], left = c[i * w + (j - 1)];
      uint8_t* bc = &b[(i - 1) * n + (j - 1)];
      if (x[i - 1] == y[j - 1]) {
        c[i * w + j] = diag + 1; *bc = ORACLE_DIAG;
      } else if (up >= left) {
        c[i * w + j] = up; *bc = ORACLE_UP;
      } else {
        c[i * w + j] = left; *bc = ORACLE_LEFT;
      }
    }
  }
  return ORACLE_OK;
}
