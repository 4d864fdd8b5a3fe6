/*
 * sfm_oracle.c -- plain FP64 CPU oracle of one time step of the discrete social
 * field pedestrian model (Yu, Zhu, Wu, Zhang, "Improved OpenCL-based
 * Implementation of Social Field Pedestrian Model").
 *
 * TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header,
 * table or constant generator with the CUDA library; the two agree only
 * through the model definition below.
 *
 * Model (the paper gives the step structure, Alg. 1 and Sec. 3.1, and names
 * the field kinds, Sec. 2, but leaves the field laws to its predecessors; the
 * laws below are this project's stated reading of them):
 *
 *   Field (superposition, Sec. 2 and sub-job k-5 of Sec. 3.1):
 *     F(c) = sum_{alive p} K_P(c - x_p; h_p) + sum_{WALL o} K_O(c - o)
 *            + sum_{EXIT e} K_E(c - e)
 *     with offsets taken as the minimum image in periodic dimensions, and every
 *     kernel zero unless 0 < max(|dx|,|dy|) <= r (square (2r+1)^2 field
 *     geometry, "7x7" <-> r = 3, Sec. 3.2 and Sec. 5).
 *     K_P(d; h) = kP |d|^aP (1 + gamma (h . d)/|d|)   (pedestrian field; the
 *                 paper's example recurrent field has k = 1, alpha = -0.5)
 *     K_O(d)    = kO |d|^aO                           (obstacles, repulsive)
 *     K_E(d)    = kE |d|^aE   with kE < 0             (openings, attractive)
 *   Guidance: D(c) = 8-connected geodesic chamfer distance through non-WALL su
 *     to the nearest EXIT su, straight step 5, diagonal step 7 (the 5-7 chamfer
 *     of Borgefors 1986); G = D / 5 su.
 *   Decision (sub-job k-2; v_max = 1 su/tick, Sec. 2): for each live p and
 *     each candidate k = 0..8 (stay + 8 neighbours), admissible iff k = 0 or
 *     the target is inside the lattice, not WALL and unoccupied at step start:
 *       E_p(k) = F(c_k) - [k>0] K_P(Delta_k; h_p) + guide_p(k)
 *       guide_p(k) = beta (D(c_k) - D(x_p)) / 5     for an exit-seeker
 *                  = -beta (Delta_k . u_goal)         for a fixed direction
 *     choice = argmin over admissible k, ties to the smallest k.
 *   Vote (sub-job k-3, enrollment container of at most 8, Sec. 3.1 s-2): each
 *     target su goes to the registrant with the smallest (prio, id), prio =
 *     SplitMix64 output (Steele, Lea, Flood 2014) counted by (seed, t, id).
 *   Commit (sub-job k-4): winners move, heading class <- move class; a winner
 *     that lands on an EXIT su leaves the lattice.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_FREE 0
#define ORC_WALL 1
#define ORC_EXIT 2
#define ORC_DINF (1 << 23)

typedef struct {
  int32_t W, H, periodic_x, periodic_y;
  int32_t r;
  int32_t pad_;
  double kP, aP, gamma, kO, aO, kE, aE, beta;
  uint64_t seed;
} orc_model;

/* candidate move offsets, class 0..8 */
static const int ODX[9] = {0, 1, 1, 0, -1, -1, -1, 0, 1};
static const int ODY[9] = {0, 0, 1, 1, 1, 0, -1, -1, -1};

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

/* Unit vector of direction class k (zero vector for k = 0). */
static void unit_dir(int k, double* ux, double* uy) {
  if (k <= 0 || k > 8) { *ux = 0.0; *uy = 0.0; return; }
  double n = sqrt((double)(ODX[k] * ODX[k] + ODY[k] * ODY[k]));
  *ux = ODX[k] / n;
  *uy = ODY[k] / n;
}

/* Field kernels of the three source kinds at offset (dx, dy) = c - source.
 * kind 0 = pedestrian with heading class hcls, 1 = WALL, 2 = EXIT. */
double orc_kernel(const orc_model* m, int kind, int dx, int dy, int hcls) {
  int adx = dx < 0 ? -dx : dx, ady = dy < 0 ? -dy : dy;
  int cheb = adx > ady ? adx : ady;
  if (cheb == 0 || cheb > m->r) return 0.0;
  double d = sqrt((double)dx * dx + (double)dy * dy);
  if (kind == ORC_WALL) return m->kO * pow(d, m->aO);
  if (kind == ORC_EXIT) return m->kE * pow(d, m->aE);
  double hx, hy;
  unit_dir(hcls, &hx, &hy);
  return m->kP * pow(d, m->aP) * (1.0 + m->gamma * (hx * dx + hy * dy) / d);
}

/* Wrap / clip a coordinate; returns 0 when it falls outside a closed side. */
static int wrap(int v, int n, int periodic, int* out) {
  if (v >= 0 && v < n) { *out = v; return 1; }
  if (!periodic) return 0;
  v %= n;
  if (v < 0) v += n;
  *out = v;
  return 1;
}

/* Per-su pedestrian index (-1 = empty).  Returns the number of conflicts
 * (two live pedestrians on one su, or one on a WALL/EXIT su or off-lattice). */
int64_t orc_occupancy(const orc_model* m, const uint8_t* cell, int32_t n, const int32_t* xy,
                      const uint8_t* alive, int32_t* occ) {
  int64_t nsu = (int64_t)m->W * m->H, bad = 0;
  for (int64_t i = 0; i < nsu; ++i) occ[i] = -1;
  for (int32_t p = 0; p < n; ++p) {
    if (alive && !alive[p]) continue;
    int x = xy[2 * p], y = xy[2 * p + 1];
    if (x < 0 || x >= m->W || y < 0 || y >= m->H) { ++bad; continue; }
    int64_t c = (int64_t)y * m->W + x;
    if (occ[c] >= 0 || (cell && cell[c] != ORC_FREE)) ++bad;
    occ[c] = p;
  }
  return bad;
}

/* ---- multi-su pedestrians (Sec. 2; Table V) ----
 * Reading: pedestrian p has odd width w_p and height h_p and occupies the
 * w_p x h_p rectangle R(x_p) of su centred on its centre su x_p (wrapped in
 * periodic dimensions).  Its field is emitted from the centre (the field
 * functions above are unchanged and read only centres).  cover[su] = p for
 * every su of p's rectangle, -1 elsewhere.  Returns the number of violations
 * (a rectangle leaving a closed lattice, overlapping another or a WALL su,
 * a centre on a non-FREE su).  w == NULL: every pedestrian is 1 x 1. */
static int rect_su(const orc_model* m, int cx, int cy, int i, int j, int64_t* out) {
  int x, y;
  if (!wrap(cx + i, m->W, m->periodic_x, &x) || !wrap(cy + j, m->H, m->periodic_y, &y)) return 0;
  *out = (int64_t)y * m->W + x;
  return 1;
}

int64_t orc_cover(const orc_model* m, const uint8_t* cell, int32_t n, const int32_t* xy,
                  const uint8_t* alive, const uint8_t* w, const uint8_t* h, int32_t* cover) {
  int64_t nsu = (int64_t)m->W * m->H, bad = 0;
  for (int64_t i = 0; i < nsu; ++i) cover[i] = -1;
  for (int32_t p = 0; p < n; ++p) {
    if (alive && !alive[p]) continue;
    int x = xy[2 * p], y = xy[2 * p + 1];
    int a = w ? w[p] / 2 : 0, b = h ? h[p] / 2 : 0;
    if (x < 0 || x >= m->W || y < 0 || y >= m->H) { ++bad; continue; }
    if (cell && cell[(int64_t)y * m->W + x] != ORC_FREE) ++bad;
    for (int j = -b; j <= b; ++j)
      for (int i = -a; i <= a; ++i) {
        int64_t s;
        if (!rect_su(m, x, y, i, j, &s)) { ++bad; continue; }
        if (cover[s] >= 0 || (cell && cell[s] == ORC_WALL)) ++bad;
        cover[s] = p;
      }
  }
  return bad;
}

/* The su p newly enters when its centre moves by move class k: R(x + D_k)
 * minus R(x).  Writes up to w + h - 1 su to out; returns the count, or -1 if
 * the moved rectangle leaves a closed lattice. */
static int entered_strip(const orc_model* m, int x, int y, int a, int b, int k, int64_t* out) {
  int dx = ODX[k], dy = ODY[k], cnt = 0;
  for (int j = -b; j <= b; ++j)
    for (int i = -a; i <= a; ++i) {
      /* (i, j) relative to the new centre; keep it unless it lies in R(x) */
      int ox = i + dx, oy = j + dy;  /* offset from the old centre */
      if (ox >= -a && ox <= a && oy >= -b && oy <= b) continue;
      int64_t s;
      if (!rect_su(m, x + dx, y + dy, i, j, &s)) return -1;
      out[cnt++] = s;
    }
  return cnt;
}

/* Field at one su c by direct superposition over its (2r+1)^2 window.
 * parts: bit 0 = WALL and EXIT sources, bit 1 = pedestrians.
 * *f receives the field, *s the sum of the terms' magnitudes. */
static void field_at(const orc_model* m, const uint8_t* cell, const int32_t* occ,
                     const uint8_t* heading, int32_t parts, int64_t c, double* f, double* s) {
  const int r = m->r;
  int cx = (int)(c % m->W), cy = (int)(c / m->W);
  double ff = 0.0, ss = 0.0;
  for (int dy = -r; dy <= r; ++dy) {
    int sy;
    if (!wrap(cy - dy, m->H, m->periodic_y, &sy)) continue;
    for (int dx = -r; dx <= r; ++dx) {
      int sx;
      if (!wrap(cx - dx, m->W, m->periodic_x, &sx)) continue;
      int64_t src = (int64_t)sy * m->W + sx;
      double term = 0.0;
      if ((parts & 1) && cell[src] == ORC_WALL) term += orc_kernel(m, ORC_WALL, dx, dy, 0);
      if ((parts & 1) && cell[src] == ORC_EXIT) term += orc_kernel(m, ORC_EXIT, dx, dy, 0);
      if ((parts & 2) && occ[src] >= 0) term += orc_kernel(m, 0, dx, dy, heading[occ[src]]);
      ff += term;
      ss += fabs(term);
    }
  }
  *f = ff;
  *s = ss;
}

/* Field at requested su (req == NULL: every su in row-major order, nreq = W*H).
 * F receives the field, S (optional) the sum of the terms' magnitudes. */
void orc_field(const orc_model* m, const uint8_t* cell, const int32_t* occ,
               const uint8_t* heading, int32_t parts, int64_t nreq, const int64_t* req,
               double* F, double* S) {
#pragma omp parallel for schedule(dynamic, 256)
  for (int64_t q = 0; q < nreq; ++q) {
    double f, s;
    field_at(m, cell, occ, heading, parts, req ? req[q] : q, &f, &s);
    F[q] = f;
    if (S) S[q] = s;
  }
}

/* ---- guidance: multi-source shortest paths with integer weights 5 / 7 ----
 * Dial's bucket-queue form of Dijkstra's algorithm (weights are small
 * integers, so a circular array of 8 buckets holds the frontier). */
typedef struct { int64_t* v; int64_t n, cap; } orc_bucket;

static void bucket_push(orc_bucket* b, int64_t x) {
  if (b->n == b->cap) {
    b->cap = b->cap ? 2 * b->cap : 1024;
    b->v = (int64_t*)realloc(b->v, (size_t)b->cap * sizeof(int64_t));
  }
  b->v[b->n++] = x;
}

int orc_guidance(const orc_model* m, const uint8_t* cell, int32_t* D) {
  const int64_t nsu = (int64_t)m->W * m->H;
  orc_bucket bk[8];
  memset(bk, 0, sizeof(bk));
  int64_t pending = 0;
  for (int64_t i = 0; i < nsu; ++i) {
    D[i] = ORC_DINF;
    if (cell[i] == ORC_EXIT) { D[i] = 0; bucket_push(&bk[0], i); ++pending; }
  }
  for (int32_t d = 0; pending > 0; ++d) {
    orc_bucket* b = &bk[d & 7];
    /* items can be appended to the current bucket only with weight 0: none */
    for (int64_t j = 0; j < b->n; ++j) {
      int64_t c = b->v[j];
      --pending;
      if (D[c] != d) continue; /* stale entry */
      int cx = (int)(c % m->W), cy = (int)(c / m->W);
      for (int k = 1; k <= 8; ++k) {
        int nx, ny;
        if (!wrap(cx + ODX[k], m->W, m->periodic_x, &nx)) continue;
        if (!wrap(cy + ODY[k], m->H, m->periodic_y, &ny)) continue;
        int64_t nb = (int64_t)ny * m->W + nx;
        if (cell[nb] == ORC_WALL) continue;
        int32_t nd = d + ((ODX[k] != 0 && ODY[k] != 0) ? 7 : 5);
        if (nd < D[nb]) {
          D[nb] = nd;
          bucket_push(&bk[nd & 7], nb);
          ++pending;
        }
      }
    }
    b->n = 0;
  }
  for (int k = 0; k < 8; ++k) free(bk[k].v);
  return 0;
}

/* ---- counter-based priority: SplitMix64 (Steele, Lea, Flood 2014) ---- */
static const uint64_t ORC_GOLDEN = 0x9e3779b97f4a7c15ULL;

uint64_t orc_mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

/* i-th output (i >= 1) of a SplitMix64 generator whose state starts at s. */
uint64_t orc_splitmix64_nth(uint64_t s, uint64_t i) { return orc_mix64(s + i * ORC_GOLDEN); }

/* Election priority of pedestrian id at step t. */
uint64_t orc_prio(uint64_t seed, int64_t t, int64_t id) {
  uint64_t st = orc_splitmix64_nth(seed, (uint64_t)t + 1);
  return orc_splitmix64_nth(st, (uint64_t)id + 1);
}

/* ---- decision (sub-job k-2) ----
 * For each requested pedestrian: E[9], the tolerance scale T[9] (sum of the
 * magnitudes of every term entering E), admissibility, and the choice.
 * Mag (optional, 9 per pedestrian): the magnitude of the energy's three
 * parts, |F(c_k)| + |own-field term| + |guidance term|, the scale of a near
 * tie (two admissible energies within 1e-5 of it).
 * Ffull/Sfull: optional full-lattice field and magnitude (row-major); when
 * NULL the field is evaluated at the candidates directly. */
void orc_decide(const orc_model* m, const uint8_t* cell, const int32_t* occ, const int32_t* xy,
                const uint8_t* heading, const uint8_t* goal, const uint8_t* alive,
                const int32_t* D, const double* Ffull, const double* Sfull, int64_t nreq,
                const int32_t* req, uint8_t* choice, double* E, double* T, uint8_t* adm,
                const int32_t* cover, const uint8_t* w, const uint8_t* h, double* Mag) {
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t q = 0; q < nreq; ++q) {
    int32_t p = req ? req[q] : (int32_t)q;
    double* e = E + 9 * q;
    double* tt = T + 9 * q;
    double* mg = Mag ? Mag + 9 * q : NULL;
    uint8_t* a = adm + 9 * q;
    for (int k = 0; k < 9; ++k) {
      e[k] = INFINITY;
      tt[k] = 0.0;
      a[k] = 0;
      if (mg) mg[k] = 0.0;
    }
    if (alive && !alive[p]) { choice[q] = 0; continue; }
    int x = xy[2 * p], y = xy[2 * p + 1];
    int64_t c0 = (int64_t)y * m->W + x;
    int64_t cand[9];
    for (int k = 0; k < 9; ++k) {
      int nx, ny;
      cand[k] = -1;
      if (!wrap(x + ODX[k], m->W, m->periodic_x, &nx)) continue;
      if (!wrap(y + ODY[k], m->H, m->periodic_y, &ny)) continue;
      int64_t c = (int64_t)ny * m->W + nx;
      if (k > 0 && !cover && (cell[c] == ORC_WALL || occ[c] >= 0)) continue;
      if (k > 0 && cover) {
        /* multi-su: every su the rectangle newly enters is inside, not WALL
           and not covered by another pedestrian at tick start */
        int64_t strip[64];
        int ns = entered_strip(m, x, y, w ? w[p] / 2 : 0, h ? h[p] / 2 : 0, k, strip);
        int ok = ns > 0;
        for (int i = 0; ok && i < ns; ++i)
          if (cell[strip[i]] == ORC_WALL || cover[strip[i]] >= 0) ok = 0;
        if (!ok) continue;
      }
      cand[k] = c;
      a[k] = 1;
    }
    double fv[9], sv[9];
    for (int k = 0; k < 9; ++k) {
      if (cand[k] < 0) continue;
      if (Ffull) {
        fv[k] = Ffull[cand[k]];
        sv[k] = Sfull ? Sfull[cand[k]] : 0.0;
      } else {
        field_at(m, cell, occ, heading, 3, cand[k], &fv[k], &sv[k]);
      }
    }
    double gx = 0.0, gy = 0.0;
    unit_dir(goal ? goal[p] : 0, &gx, &gy);
    int best = -1;
    for (int k = 0; k < 9; ++k) {
      if (cand[k] < 0) continue;
      double own = (k > 0) ? orc_kernel(m, 0, ODX[k], ODY[k], heading[p]) : 0.0;
      double g;
      if (!goal || goal[p] == 0)
        g = m->beta * (double)(D[cand[k]] - D[c0]) / 5.0;
      else
        g = -m->beta * (ODX[k] * gx + ODY[k] * gy);
      e[k] = fv[k] - own + g;
      tt[k] = sv[k] + fabs(own) + fabs(g);
      if (mg) mg[k] = fabs(fv[k]) + fabs(own) + fabs(g);
      if (best < 0 || e[k] < e[best]) best = k;
    }
    choice[q] = (uint8_t)(best < 0 ? 0 : best);
  }
}

/* ---- vote (sub-job k-3) ---- */
typedef struct { int64_t target; uint64_t prio; int32_t id, p; } orc_reg;

static int reg_cmp(const void* a, const void* b) {
  const orc_reg* x = (const orc_reg*)a;
  const orc_reg* y = (const orc_reg*)b;
  if (x->target != y->target) return x->target < y->target ? -1 : 1;
  if (x->prio != y->prio) return x->prio < y->prio ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id);
}

/* won[p] = 1 for the winner of each contested su; returns the number of
 * registrants of the most contested su (the enrollment bound says <= 8).
 * Pedestrian p is numbered ids[p] (its priority and tie-break), or p when
 * ids is NULL: a lattice that is one band of a larger one numbers its
 * pedestrians, ghosts included, as the larger lattice does. */
int32_t orc_vote_numbered(const orc_model* m, int64_t t, int32_t n, const int32_t* xy,
                          const uint8_t* alive, const uint8_t* choice, const int32_t* ids,
                          uint8_t* won) {
  orc_reg* regs = (orc_reg*)malloc(sizeof(orc_reg) * (size_t)(n > 0 ? n : 1));
  int32_t nr = 0;
  for (int32_t p = 0; p < n; ++p) {
    won[p] = 0;
    if ((alive && !alive[p]) || choice[p] == 0) continue;
    int nx = 0, ny = 0;
    if (!wrap(xy[2 * p] + ODX[choice[p]], m->W, m->periodic_x, &nx) ||
        !wrap(xy[2 * p + 1] + ODY[choice[p]], m->H, m->periodic_y, &ny))
      continue; /* an off-lattice target is never admissible */
    regs[nr].target = (int64_t)ny * m->W + nx;
    regs[nr].prio = orc_prio(m->seed, t, ids ? ids[p] : p);
    regs[nr].id = ids ? ids[p] : p;
    regs[nr].p = p;
    ++nr;
  }
  qsort(regs, (size_t)nr, sizeof(orc_reg), reg_cmp);
  int32_t maxc = 0;
  for (int32_t i = 0; i < nr;) {
    int32_t j = i;
    while (j < nr && regs[j].target == regs[i].target) ++j;
    won[regs[i].p] = 1;
    if (j - i > maxc) maxc = j - i;
    i = j;
  }
  free(regs);
  return maxc;
}

int32_t orc_vote(const orc_model* m, int64_t t, int32_t n, const int32_t* xy,
                 const uint8_t* alive, const uint8_t* choice, uint8_t* won) {
  return orc_vote_numbered(m, t, n, xy, alive, choice, NULL, won);
}

/* Vote with multi-su pedestrians: a mover claims the su its rectangle newly
 * enters; it wins iff its (prio, id) is the smallest among the claimants of
 * every su it claims, i.e. smaller than that of every mover whose claim
 * intersects its own.  With 1 x 1 pedestrians a claim is the target su and
 * this is orc_vote.  Returns the most claimants of one su. */
typedef struct { int64_t su; uint64_t prio; int32_t id; } orc_claim;

static int claim_cmp(const void* a, const void* b) {
  const orc_claim* x = (const orc_claim*)a;
  const orc_claim* y = (const orc_claim*)b;
  if (x->su != y->su) return x->su < y->su ? -1 : 1;
  if (x->prio != y->prio) return x->prio < y->prio ? -1 : 1;
  return x->id < y->id ? -1 : (x->id > y->id);
}

int32_t orc_vote_sized(const orc_model* m, int64_t t, int32_t n, const int32_t* xy,
                       const uint8_t* alive, const uint8_t* choice, const uint8_t* w,
                       const uint8_t* h, uint8_t* won) {
  size_t cap = 16, nc = 0;
  orc_claim* cl = (orc_claim*)malloc(sizeof(orc_claim) * cap);
  for (int32_t p = 0; p < n; ++p) {
    won[p] = 0;
    if ((alive && !alive[p]) || choice[p] == 0) continue;
    int64_t strip[64];
    int ns = entered_strip(m, xy[2 * p], xy[2 * p + 1], w[p] / 2, h[p] / 2, choice[p], strip);
    if (ns <= 0) continue;
    won[p] = 1;  /* until a claimant with a smaller (prio, id) shares a su */
    uint64_t pr = orc_prio(m->seed, t, p);
    for (int i = 0; i < ns; ++i) {
      if (nc == cap) {
        cap *= 2;
        cl = (orc_claim*)realloc(cl, sizeof(orc_claim) * cap);
      }
      cl[nc].su = strip[i];
      cl[nc].prio = pr;
      cl[nc].id = p;
      ++nc;
    }
  }
  qsort(cl, nc, sizeof(orc_claim), claim_cmp);
  int32_t maxc = 0;
  for (size_t i = 0; i < nc;) {
    size_t j = i;
    while (j < nc && cl[j].su == cl[i].su) ++j;
    for (size_t q = i + 1; q < j; ++q) won[cl[q].id] = 0;
    if ((int32_t)(j - i) > maxc) maxc = (int32_t)(j - i);
    i = j;
  }
  free(cl);
  return maxc;
}

/* ---- commit (sub-job k-4) ----  returns the number that left via exits */
int32_t orc_commit(const orc_model* m, const uint8_t* cell, int32_t n, int32_t* xy,
                   uint8_t* heading, uint8_t* alive, const uint8_t* choice, const uint8_t* won,
                   const uint8_t* w, const uint8_t* h) {
  int32_t left = 0;
  for (int32_t p = 0; p < n; ++p) {
    if ((alive && !alive[p]) || !won[p]) continue;
    int k = choice[p];
    int nx = 0, ny = 0;
    if (!wrap(xy[2 * p] + ODX[k], m->W, m->periodic_x, &nx) ||
        !wrap(xy[2 * p + 1] + ODY[k], m->H, m->periodic_y, &ny))
      continue;
    xy[2 * p] = nx;
    xy[2 * p + 1] = ny;
    heading[p] = (uint8_t)k;
    /* it leaves when it steps onto an EXIT su: its centre (1 x 1), or for a
       multi-su pedestrian any su of its new rectangle */
    int out = cell[(int64_t)ny * m->W + nx] == ORC_EXIT;
    const int a = w ? w[p] / 2 : 0, b = h ? h[p] / 2 : 0;
    for (int j = -b; !out && j <= b; ++j)
      for (int i = -a; !out && i <= a; ++i) {
        int64_t s;
        if (rect_su(m, nx, ny, i, j, &s) && cell[s] == ORC_EXIT) out = 1;
      }
    if (out) {
      alive[p] = 0;
      ++left;
    }
  }
  return left;
}

/* ---- walk period (Sec. 2) ----
 * The paper adopts walk periods from its predecessor to vary walking speeds
 * under v_max = 1 su per tick, without stating the rule.  Reading: pedestrian
 * p has a period P_p >= 1 and a phase 0 <= phase_p < P_p, and may move only
 * on ticks t with t mod P_p = phase_p; on other ticks it stays (choice 0), so
 * it registers nowhere and keeps its su.  P = 1 everywhere is the plain
 * model.  period == NULL: every pedestrian is active. */
void orc_gate_periods(int64_t t, int32_t n, const uint8_t* period, const uint8_t* phase,
                      uint8_t* choice) {
  if (!period) return;
  for (int32_t p = 0; p < n; ++p)
    if (t % (int64_t)period[p] != (int64_t)phase[p]) choice[p] = 0;
}

/* ---- one full step (Alg. 1): decide all, vote, commit ----
 * D must hold the guidance distances; occ scratch of W*H int32; choice and won
 * receive the per-pedestrian results; period/phase as orc_gate_periods (NULL:
 * all active); w/h the pedestrians' rectangles (NULL: 1 x 1).  Returns the
 * number that left. */
int32_t orc_step(const orc_model* m, const uint8_t* cell, const int32_t* D, int64_t t, int32_t n,
                 int32_t* xy, uint8_t* heading, const uint8_t* goal, uint8_t* alive, int32_t* occ,
                 uint8_t* choice, uint8_t* won, const uint8_t* period, const uint8_t* phase,
                 const uint8_t* w, const uint8_t* h) {
  orc_occupancy(m, cell, n, xy, alive, occ);
  double* E = (double*)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
  double* T = (double*)malloc(sizeof(double) * 9 * (size_t)(n > 0 ? n : 1));
  uint8_t* adm = (uint8_t*)malloc(9 * (size_t)(n > 0 ? n : 1));
  int32_t* cover = NULL;
  if (w) {
    cover = (int32_t*)malloc(sizeof(int32_t) * (size_t)m->W * m->H);
    orc_cover(m, cell, n, xy, alive, w, h, cover);
  }
  orc_decide(m, cell, occ, xy, heading, goal, alive, D, NULL, NULL, n, NULL, choice, E, T, adm,
             cover, w, h, NULL);
  orc_gate_periods(t, n, period, phase, choice);
  if (w)
    orc_vote_sized(m, t, n, xy, alive, choice, w, h, won);
  else
    orc_vote(m, t, n, xy, alive, choice, won);
  free(cover);
  int32_t left = orc_commit(m, cell, n, xy, heading, alive, choice, won, w, h);
  free(E);
  free(T);
  free(adm);
  return left;
}
