/*
 * Multi-threaded CPU oracle — TEST INFRASTRUCTURE ONLY (tests and the benchmark's CPU-baseline legs).
 *
 * The paper's parallel algorithm (Dash & Nayak, §II.A-B) on host threads: the table of LCS-length (§I.C) is cut
 * into blocks of columns ("block sections"), one per processor; every processor fills its block with the same
 * recurrence and tie-break as the serial oracle (DIAG on a match; else UP when c[i-1,j] >= c[i,j-1], else LEFT),
 * and the root gathers the result: the length c[m,n] and, through Print-LCS (§I.D) on the gathered table b, the
 * LCS string. The paper does not say how the blocks wait for each other; a cell needs its left neighbour, so
 * processor p fills rows [r0, r1) of its block only after processor p-1 has finished the same rows (a wavefront
 * over row chunks). Every value is the serial oracle's; only the order in which independent cells are filled
 * differs.
 *
 * Storage: b at one byte per cell (processors write disjoint bytes), c as rolling rows inside each block plus
 * the last column of every block for all rows (read by the block to its right). The traceback is meant for the
 * paper's problem sizes (Table 1: up to 10000 x 1500) and test cases; oracle_lcs_length_par keeps no b and runs at
 * any size whose edge columns fit (threads * m words).
 */
#include <pthread.h>
#include <sched.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { PAR_DIAG = 1, PAR_UP = 2, PAR_LEFT = 3 };
enum { PAR_OK = 0, PAR_ERR_NOMEM = -1, PAR_ERR_CAPACITY = -2, PAR_ERR_INVALID = -3 };

typedef struct {
  const uint8_t* x;
  const uint8_t* y;
  uint64_t m, n, rows_per_chunk;
  int nproc;
  uint64_t* j0;               /* block p covers columns j0[p] .. j0[p+1]-1 (1-based) */
  uint32_t* edge;             /* edge[p * (m + 1) + i] = c[i, j0[p+1] - 1] */
  uint8_t* b;                 /* b[(i - 1) * n + (j - 1)], or NULL for the length only */
  volatile uint64_t* done;    /* done[p] = rows of block p finished (published with release order) */
} ParShared;

typedef struct {
  ParShared* s;
  int p;
  int rc;
} ParTask;

static void* par_fill_block(void* arg) {
  ParTask* t = (ParTask*)arg;
  ParShared* s = t->s;
  const int p = t->p;
  const uint64_t ja = s->j0[p], jb = s->j0[p + 1], w = jb - ja;
  uint32_t* prev = (uint32_t*)calloc(w + 1, sizeof(uint32_t)); /* prev[k] = c[i-1, ja-1+k] */
  uint32_t* cur = (uint32_t*)calloc(w + 1, sizeof(uint32_t));
  if (!prev || !cur) {
    free(prev);
    free(cur);
    t->rc = PAR_ERR_NOMEM;
    /* publish every row so that the block to the right does not wait forever; its values are unused */
    __atomic_store_n(&s->done[p], s->m, __ATOMIC_RELEASE);
    return NULL;
  }
  const uint32_t* left = p > 0 ? s->edge + (uint64_t)(p - 1) * (s->m + 1) : NULL;
  uint32_t* mine = s->edge + (uint64_t)p * (s->m + 1);
  mine[0] = 0;
  for (uint64_t r0 = 1; r0 <= s->m; r0 += s->rows_per_chunk) {
    const uint64_t r1 = r0 + s->rows_per_chunk <= s->m + 1 ? r0 + s->rows_per_chunk : s->m + 1;
    if (p > 0)
      while (__atomic_load_n(&s->done[p - 1], __ATOMIC_ACQUIRE) < r1 - 1) sched_yield();
    for (uint64_t i = r0; i < r1; ++i) {
      cur[0] = left ? left[i] : 0;   /* c[i, ja-1] */
      prev[0] = left ? left[i - 1] : 0; /* c[i-1, ja-1] */
      const uint8_t xi = s->x[i - 1];
      if (s->b) {
        for (uint64_t k = 1; k <= w; ++k) {
          const uint64_t j = ja - 1 + k;
          uint8_t* bc = &s->b[(i - 1) * s->n + (j - 1)];
          if (xi == s->y[j - 1]) {
            cur[k] = prev[k - 1] + 1;
            *bc = PAR_DIAG;
          } else if (prev[k] >= cur[k - 1]) {
            cur[k] = prev[k];
            *bc = PAR_UP;
          } else {
            cur[k] = cur[k - 1];
            *bc = PAR_LEFT;
          }
        }
      } else {  /* the same recurrence without the arrows */
        for (uint64_t k = 1; k <= w; ++k) {
          const uint64_t j = ja - 1 + k;
          if (xi == s->y[j - 1]) {
            cur[k] = prev[k - 1] + 1;
          } else if (prev[k] >= cur[k - 1]) {
            cur[k] = prev[k];
          } else {
            cur[k] = cur[k - 1];
          }
        }
      }
      mine[i] = cur[w];
      uint32_t* tmp = prev;
      prev = cur;
      cur = tmp;
    }
    __atomic_store_n(&s->done[p], r1 - 1, __ATOMIC_RELEASE);
  }
  free(prev);
  free(cur);
  t->rc = PAR_OK;
  return NULL;
}

/* LCS-length (§I.C) with table b filled by `threads` processors, then Print-LCS (§I.D). Same outputs and return
 * codes as oracle_lcs_traceback. */
int oracle_lcs_traceback_par(const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, uint8_t* out,
                             uint64_t out_cap, uint64_t* out_len, int threads) {
  if (!out_len || threads < 1) return PAR_ERR_INVALID;
  *out_len = 0;
  if (m == 0 || n == 0) return PAR_OK;
  const uint64_t cells = m * n;
  if (cells / m != n) return PAR_ERR_INVALID;
  int np = threads;
  if ((uint64_t)np > n) np = (int)n;
  ParShared s;
  memset(&s, 0, sizeof(s));
  s.x = x;
  s.y = y;
  s.m = m;
  s.n = n;
  s.nproc = np;
  s.rows_per_chunk = m < 64 ? m : 64;
  s.j0 = (uint64_t*)malloc((size_t)(np + 1) * sizeof(uint64_t));
  s.edge = (uint32_t*)calloc((size_t)np * (m + 1), sizeof(uint32_t));
  s.b = (uint8_t*)malloc(cells);
  s.done = (volatile uint64_t*)calloc((size_t)np, sizeof(uint64_t));
  ParTask* tasks = (ParTask*)calloc((size_t)np, sizeof(ParTask));
  pthread_t* tid = (pthread_t*)calloc((size_t)np, sizeof(pthread_t));
  uint8_t* rev = (uint8_t*)malloc(m < n ? m : n);
  int rc = PAR_OK;
  if (!s.j0 || !s.edge || !s.b || !s.done || !tasks || !tid || !rev) rc = PAR_ERR_NOMEM;
  if (rc == PAR_OK) {
    for (int p = 0; p <= np; ++p) s.j0[p] = 1 + (n * (uint64_t)p) / (uint64_t)np; /* near-equal blocks */
    int started = 0;
    for (int p = 0; p < np; ++p) {
      tasks[p].s = &s;
      tasks[p].p = p;
      tasks[p].rc = PAR_OK;
      if (p == 0) continue; /* the root fills block 0 itself */
      if (pthread_create(&tid[p], NULL, par_fill_block, &tasks[p]) != 0) break;
      started = p;
    }
    if (started == np - 1) {
      par_fill_block(&tasks[0]);
    } else {
      /* thread creation failed: fill the remaining blocks on this thread, in order */
      rc = PAR_OK;
      for (int p = 0; p < np; ++p)
        if (p == 0 || p > started) par_fill_block(&tasks[p]);
    }
    for (int p = 1; p <= started; ++p) pthread_join(tid[p], NULL);
    for (int p = 0; p < np; ++p)
      if (tasks[p].rc != PAR_OK) rc = tasks[p].rc;
  }
  uint64_t len = 0, k = 0;
  if (rc == PAR_OK) {
    len = s.edge[(uint64_t)(np - 1) * (m + 1) + m]; /* c[m, n] */
    uint64_t i = m, j = n;
    while (i > 0 && j > 0) {
      const uint8_t d = s.b[(i - 1) * n + (j - 1)];
      if (d == PAR_DIAG) {
        rev[k++] = x[i - 1];
        --i;
        --j;
      } else if (d == PAR_UP) {
        --i;
      } else {
        --j;
      }
    }
    *out_len = len;
    if (k != len) rc = PAR_ERR_INVALID;
    else if (out_cap < len) rc = PAR_ERR_CAPACITY;
    else
      for (uint64_t t = 0; t < len; ++t) out[t] = rev[len - 1 - t];
  }
  free(s.j0);
  free(s.edge);
  free(s.b);
  free((void*)s.done);
  free(tasks);
  free(tid);
  free(rev);
  return rc;
}

/* LCS-length (§I.C), length only, filled by `threads` processors in column blocks as above; c[m, n], or UINT64_MAX
 * when memory runs out. The row arrays and the blocks' edge columns take O(threads * m + n) words, so this runs
 * at sizes where the table b could not be stored. */
uint64_t oracle_lcs_length_par(const uint8_t* x, uint64_t m, const uint8_t* y, uint64_t n, int threads) {
  if (m == 0 || n == 0) return 0;
  if (threads < 1) threads = 1;
  int np = threads;
  if ((uint64_t)np > n) np = (int)n;
  ParShared s;
  memset(&s, 0, sizeof(s));
  s.x = x;
  s.y = y;
  s.m = m;
  s.n = n;
  s.nproc = np;
  s.rows_per_chunk = m < 256 ? m : 256;
  s.b = NULL;
  s.j0 = (uint64_t*)malloc((size_t)(np + 1) * sizeof(uint64_t));
  s.edge = (uint32_t*)calloc((size_t)np * (m + 1), sizeof(uint32_t));
  s.done = (volatile uint64_t*)calloc((size_t)np, sizeof(uint64_t));
  ParTask* tasks = (ParTask*)calloc((size_t)np, sizeof(ParTask));
  pthread_t* tid = (pthread_t*)calloc((size_t)np, sizeof(pthread_t));
  uint64_t len = UINT64_MAX;
  if (s.j0 && s.edge && s.done && tasks && tid) {
    for (int p = 0; p <= np; ++p) s.j0[p] = 1 + (n * (uint64_t)p) / (uint64_t)np;
    int started = 0;
    for (int p = 0; p < np; ++p) {
      tasks[p].s = &s;
      tasks[p].p = p;
      tasks[p].rc = PAR_OK;
      if (p == 0) continue;
      if (pthread_create(&tid[p], NULL, par_fill_block, &tasks[p]) != 0) break;
      started = p;
    }
    par_fill_block(&tasks[0]);
    for (int p = started + 1; p < np; ++p) par_fill_block(&tasks[p]); /* blocks whose thread did not start */
    for (int p = 1; p <= started; ++p) pthread_join(tid[p], NULL);
    int ok = 1;
    for (int p = 0; p < np; ++p)
      if (tasks[p].rc != PAR_OK) ok = 0;
    if (ok) len = s.edge[(uint64_t)(np - 1) * (m + 1) + m];
  }
  free(s.j0);
  free(s.edge);
  free((void*)s.done);
  free(tasks);
  free(tid);
  return len;
}
