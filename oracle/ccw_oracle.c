/*
 * ccw_oracle.c -- plain, slow, single-threaded CPU oracle of the CCWSIM
 * best-match search (Bavandsavadkoohi et al., "CCWSIM", arXiv 2404.00441).
 *
 * TEST INFRASTRUCTURE ONLY. Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library. It shares no code, header,
 * table or constant with the CUDA library, and the CUDA library never calls
 * it.
 *
 * Everything is integer (int64) arithmetic, which is exact for the scaled
 * Haar transform used here. Each function states the passage of the paper it
 * follows. Readings of passages the paper leaves open:
 *   - Haar normalisation: the "scaled" integer Haar (lo = a+b, hi = a-b) is
 *     used; it differs from the orthonormal one of Sec. 3.1 / Sec. 4.2 by the
 *     positive factor 2^(-d/2) per level, so every CCW ranking is the same.
 *     The orthonormal transform is also provided (orc_dwt_orth) for the
 *     tolerance tests.
 *   - Categorical score: the CCW equation of Sec. 4.3 is applied to the
 *     indicator image of every facies and summed ("one-hot", score_mode 0);
 *     score_mode 1 applies it literally to the facies codes.
 *   - Candidates are the positions of the level-J approximation grid
 *     (decimated by 2^J), as in the size example of Sec. 4.3.
 *   - Top-K order: (hard-data mismatches ascending, score descending,
 *     candidate index ascending); the draw is j = floor(u * K / 2^32) with u
 *     the first Philox4x32-10 word of counter (r, p, 0, 0), key = seed.
 *   - A patch whose data event is empty takes a uniform candidate
 *     floor(u * P_c / 2^32) (Algorithm 1, "select randomly a patch").
 *   - Paste overwrites the whole template, then hard data are re-imposed.
 *   - Path randomisation mirrors the patch lattice (the raster starts from
 *     another corner); training-image patterns are never mirrored.
 *   - Non-causal conditioning (Sec. 4.4, the conditional scheme that the
 *     paper only sketches): the template grown by E cells along the forward
 *     directions of the path is the "virtual template"; the hard data in it
 *     but outside the template add to the mismatch count, a datum whose TI
 *     position falls outside the TI counting as a mismatch. The score and
 *     the empty-event rule use the template alone.
 *   - All-shift (polyphase) candidates, an option: every fine origin c of
 *     the cropped TI with c + T <= n on every axis instead of the multiples
 *     of s (decimation keeps one position in s^d per level, Sec. 3.2); the
 *     level-J approximation of the window at c is its s^d block sums, the
 *     ranking index is c's raster index over the fine candidate grid and the
 *     pasted pattern is the TI crop at c.
 *   - Minimum-error boundary cut (the image-quilting paste of Sec. 2, 2D):
 *     in the path frame, a vertical cut through the left overlap strip and
 *     a horizontal one through the top strip, each the cheapest 8-connected
 *     path over the 0/1 disagreements between the grid and the new pattern
 *     (ties to the lower column); the pattern replaces a simulated cell only
 *     on the far side of both cuts.
 *
 * Array convention: x fastest; dims n[3] = {nx, ny, nz} with nz = 1 in 2D.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_OK 0
#define ORC_EINVAL (-1)
#define ORC_ENOMEM (-2)
#define UNKNOWN 255u

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random numbers: */
/* as easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplications,  */
/* the key bumped by the Weyl constants between rounds.                      */
/* ------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2],
                       uint32_t out[4]) {
  const uint32_t m0 = 0xD2511F53u, m1 = 0xCD9E8D57u;
  const uint32_t w0 = 0x9E3779B9u, w1 = 0xBB67AE85u;
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += w0;
      k1 += w1;
    }
    uint64_t p0 = (uint64_t)m0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)m1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

/* n blocks of Philox4x32-10 under one key: ctr and out are [n][4]. */
void orc_philox_many(int64_t n, const uint32_t* ctr, const uint32_t key[2], uint32_t* out) {
  for (int64_t i = 0; i < n; ++i) orc_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

static uint32_t draw_u32(uint64_t seed, uint32_t a, uint32_t b, uint32_t purpose) {
  uint32_t ctr[4] = {a, b, purpose, 0u};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint32_t out[4];
  orc_philox4x32_10(ctr, key, out);
  return out[0];
}

/* uniform index in [0, n) by multiply-shift */
static int64_t scale_u32(uint32_t u, int64_t n) {
  return (int64_t)(((uint64_t)u * (uint64_t)n) >> 32);
}

/* ------------------------------------------------------------------------ */
/* Haar DWT (Sec. 3.1: filter rows, downsample, filter columns, downsample;  */
/* Haar scaling/wavelet functions of Sec. 4.2). One level splits an array   */
/* into 2^d sub-bands; band index b has bit a set when the band is the       */
/* high-pass output along axis a (b = 0 is the approximation).               */
/* ------------------------------------------------------------------------ */
static int64_t vol3(const int64_t n[3]) { return n[0] * n[1] * n[2]; }

/* Split `src` (dims n) along axis `a` into lo/hi halves (dims n with n[a]/2). */
static void split_axis_i64(const int64_t* src, const int64_t n[3], int a,
                           int64_t* lo, int64_t* hi) {
  int64_t m[3] = {n[0], n[1], n[2]};
  m[a] /= 2;
  for (int64_t z = 0; z < m[2]; ++z)
    for (int64_t y = 0; y < m[1]; ++y)
      for (int64_t x = 0; x < m[0]; ++x) {
        int64_t i0[3] = {x, y, z}, i1[3] = {x, y, z};
        i0[a] = 2 * i0[a];
        i1[a] = 2 * i1[a] + 1;
        int64_t s0 = src[i0[0] + n[0] * (i0[1] + n[1] * i0[2])];
        int64_t s1 = src[i1[0] + n[0] * (i1[1] + n[1] * i1[2])];
        int64_t o = x + m[0] * (y + m[1] * z);
        lo[o] = s0 + s1;
        hi[o] = s0 - s1;
      }
}

/* Inverse of split_axis_i64: x_{2i} = (lo+hi)/2, x_{2i+1} = (lo-hi)/2. */
static int merge_axis_i64(const int64_t* lo, const int64_t* hi, const int64_t m[3],
                          int a, int64_t* dst) {
  int64_t n[3] = {m[0], m[1], m[2]};
  n[a] *= 2;
  for (int64_t z = 0; z < m[2]; ++z)
    for (int64_t y = 0; y < m[1]; ++y)
      for (int64_t x = 0; x < m[0]; ++x) {
        int64_t o = x + m[0] * (y + m[1] * z);
        int64_t sum = lo[o] + hi[o], dif = lo[o] - hi[o];
        if ((sum & 1) != 0) return ORC_EINVAL; /* not a scaled-Haar pyramid */
        int64_t i0[3] = {x, y, z}, i1[3] = {x, y, z};
        i0[a] = 2 * i0[a];
        i1[a] = 2 * i1[a] + 1;
        dst[i0[0] + n[0] * (i0[1] + n[1] * i0[2])] = sum / 2;
        dst[i1[0] + n[0] * (i1[1] + n[1] * i1[2])] = dif / 2;
      }
  return ORC_OK;
}

/* Offset of detail band (j, b), 1 <= j <= J, 1 <= b < 2^d, in the pyramid
 * layout used by orc_dwt: level 1 bands first, then level 2, ..., and the
 * level-J approximation last. */
static int64_t pyr_band_offset(int ndim, const int64_t n[3], int j, int b) {
  int nb = (1 << ndim) - 1;
  int64_t off = 0;
  for (int jj = 1; jj < j; ++jj) {
    int64_t v = 1;
    for (int a = 0; a < ndim; ++a) v *= n[a] >> jj;
    off += nb * v;
  }
  int64_t vj = 1;
  for (int a = 0; a < ndim; ++a) vj *= n[a] >> j;
  return off + (int64_t)(b - 1) * vj;
}

static int64_t pyr_approx_offset(int ndim, const int64_t n[3], int J) {
  return pyr_band_offset(ndim, n, J + 1, 1);
}

/* J-level scaled Haar DWT of an integer array (every n[a] divisible by 2^J
 * for a < ndim). Output layout: for j = 1..J the 2^d - 1 detail bands of
 * level j (dims n/2^j each, band b = 1..2^d-1), then the approximation cA_J
 * (dims n/2^J). The output has exactly prod(n) entries. */
int orc_dwt(const int64_t* x, int ndim, const int32_t dims[3], int J, int64_t* pyr) {
  if (ndim < 1 || ndim > 3 || J < 0) return ORC_EINVAL;
  int64_t n[3] = {dims[0], ndim > 1 ? dims[1] : 1, ndim > 2 ? dims[2] : 1};
  for (int a = 0; a < ndim; ++a)
    if (n[a] <= 0 || (n[a] % ((int64_t)1 << J)) != 0) return ORC_EINVAL;
  int64_t total = vol3(n);
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * total);
  int64_t* bands = (int64_t*)malloc(sizeof(int64_t) * total);
  int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * total);
  if (!cur || !bands || !tmp) {
    free(cur); free(bands); free(tmp);
    return ORC_ENOMEM;
  }
  memcpy(cur, x, sizeof(int64_t) * total);
  int64_t m[3] = {n[0], n[1], n[2]};
  for (int j = 1; j <= J; ++j) {
    /* bands[b] holds sub-band b; start with one band (the input) */
    int64_t bvol = vol3(m);
    memcpy(bands, cur, sizeof(int64_t) * bvol);
    int64_t bm[3] = {m[0], m[1], m[2]};
    int nbands = 1;
    for (int a = 0; a < ndim; ++a) {
      int64_t half = bvol / 2;
      /* split every existing band b along axis a into b (lo), b|(1<<a) (hi) */
      for (int b = 0; b < nbands; ++b) {
        split_axis_i64(bands + (int64_t)b * bvol, bm, a, tmp + (int64_t)b * half,
                       tmp + (int64_t)(b + nbands) * half);
      }
      /* with nbands = 2^a, the hi half of band b lands at b + 2^a, i.e. at
       * the index of b with bit a set: tmp is already in band order */
      memcpy(bands, tmp, sizeof(int64_t) * half * 2 * nbands);
      bm[a] /= 2;
      bvol = half;
      nbands *= 2;
    }
    for (int b = 1; b < nbands; ++b)
      memcpy(pyr + pyr_band_offset(ndim, n, j, b), bands + (int64_t)b * bvol,
             sizeof(int64_t) * bvol);
    memcpy(cur, bands, sizeof(int64_t) * bvol); /* band 0 = approximation */
    for (int a = 0; a < ndim; ++a) m[a] /= 2;
  }
  memcpy(pyr + pyr_approx_offset(ndim, n, J), cur, sizeof(int64_t) * vol3(m));
  free(cur); free(bands); free(tmp);
  return ORC_OK;
}

/* Inverse of orc_dwt (the Inverse-DWT of Sec. 3.1 / Algorithm 1). */
int orc_idwt(const int64_t* pyr, int ndim, const int32_t dims[3], int J, int64_t* x) {
  if (ndim < 1 || ndim > 3 || J < 0) return ORC_EINVAL;
  int64_t n[3] = {dims[0], ndim > 1 ? dims[1] : 1, ndim > 2 ? dims[2] : 1};
  for (int a = 0; a < ndim; ++a)
    if (n[a] <= 0 || (n[a] % ((int64_t)1 << J)) != 0) return ORC_EINVAL;
  int64_t total = vol3(n);
  int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * total);
  int64_t* bands = (int64_t*)malloc(sizeof(int64_t) * total);
  int64_t* tmp = (int64_t*)malloc(sizeof(int64_t) * total);
  if (!cur || !bands || !tmp) {
    free(cur); free(bands); free(tmp);
    return ORC_ENOMEM;
  }
  int64_t m[3] = {n[0], n[1], n[2]};
  for (int a = 0; a < ndim; ++a) m[a] >>= J;
  memcpy(cur, pyr + pyr_approx_offset(ndim, n, J), sizeof(int64_t) * vol3(m));
  int rc = ORC_OK;
  for (int j = J; j >= 1 && rc == ORC_OK; --j) {
    int nb = 1 << ndim;
    int64_t bvol = vol3(m);
    memcpy(bands, cur, sizeof(int64_t) * bvol);
    for (int b = 1; b < nb; ++b)
      memcpy(bands + (int64_t)b * bvol, pyr + pyr_band_offset(ndim, n, j, b),
             sizeof(int64_t) * bvol);
    int64_t bm[3] = {m[0], m[1], m[2]};
    /* undo the axis splits in reverse order: last axis first */
    int nbands = nb;
    for (int a = ndim - 1; a >= 0 && rc == ORC_OK; --a) {
      int half_n = nbands / 2;
      int64_t ovol = bvol * 2;
      int64_t om[3] = {bm[0], bm[1], bm[2]};
      om[a] *= 2;
      for (int b = 0; b < half_n; ++b) {
        /* axes above a are merged already, so the band index keeps bits
         * 0..a: band b (bit a clear) pairs with its hi partner b | 2^a */
        int lo_i = b, hi_i = b | (1 << a);
        rc = merge_axis_i64(bands + (int64_t)lo_i * bvol, bands + (int64_t)hi_i * bvol, bm,
                            a, tmp + (int64_t)b * ovol);
        if (rc != ORC_OK) break;
      }
      memcpy(bands, tmp, sizeof(int64_t) * ovol * (int64_t)(1 << a));
      bm[a] = om[a];
      bvol = ovol;
      nbands = 1 << a;
    }
    memcpy(cur, bands, sizeof(int64_t) * bvol);
    for (int a = 0; a < ndim; ++a) m[a] *= 2;
  }
  if (rc == ORC_OK) memcpy(x, cur, sizeof(int64_t) * total);
  free(cur); free(bands); free(tmp);
  return rc;
}

/* Orthonormal Haar (filters (1, 1)/sqrt2 and (1, -1)/sqrt2, Sec. 3.1), in
 * fp64: the same band layout as orc_dwt. Used for the tolerance tests. */
int orc_dwt_orth(const double* x, int ndim, const int32_t dims[3], int J, double* pyr) {
  if (ndim < 1 || ndim > 3 || J < 0) return ORC_EINVAL;
  int64_t n[3] = {dims[0], ndim > 1 ? dims[1] : 1, ndim > 2 ? dims[2] : 1};
  for (int a = 0; a < ndim; ++a)
    if (n[a] <= 0 || (n[a] % ((int64_t)1 << J)) != 0) return ORC_EINVAL;
  const double r = 0.70710678118654752440;
  int64_t total = vol3(n);
  double* cur = (double*)malloc(sizeof(double) * total);
  double* bands = (double*)malloc(sizeof(double) * total);
  double* tmp = (double*)malloc(sizeof(double) * total);
  if (!cur || !bands || !tmp) {
    free(cur); free(bands); free(tmp);
    return ORC_ENOMEM;
  }
  memcpy(cur, x, sizeof(double) * total);
  int64_t m[3] = {n[0], n[1], n[2]};
  for (int j = 1; j <= J; ++j) {
    int64_t bvol = vol3(m);
    memcpy(bands, cur, sizeof(double) * bvol);
    int64_t bm[3] = {m[0], m[1], m[2]};
    int nbands = 1;
    for (int a = 0; a < ndim; ++a) {
      int64_t half = bvol / 2;
      int64_t hm[3] = {bm[0], bm[1], bm[2]};
      hm[a] /= 2;
      for (int b = 0; b < nbands; ++b) {
        const double* src = bands + (int64_t)b * bvol;
        double* lo = tmp + (int64_t)b * half;
        double* hi = tmp + (int64_t)(b + nbands) * half;
        for (int64_t z = 0; z < hm[2]; ++z)
          for (int64_t y = 0; y < hm[1]; ++y)
            for (int64_t xx = 0; xx < hm[0]; ++xx) {
              int64_t i0[3] = {xx, y, z}, i1[3] = {xx, y, z};
              i0[a] = 2 * i0[a];
              i1[a] = 2 * i1[a] + 1;
              double s0 = src[i0[0] + bm[0] * (i0[1] + bm[1] * i0[2])];
              double s1 = src[i1[0] + bm[0] * (i1[1] + bm[1] * i1[2])];
              int64_t o = xx + hm[0] * (y + hm[1] * z);
              lo[o] = (s0 + s1) * r;
              hi[o] = (s0 - s1) * r;
            }
      }
      memcpy(bands, tmp, sizeof(double) * half * 2 * nbands);
      bm[a] /= 2;
      bvol = half;
      nbands *= 2;
    }
    for (int b = 1; b < nbands; ++b)
      memcpy(pyr + pyr_band_offset(ndim, n, j, b), bands + (int64_t)b * bvol,
             sizeof(double) * bvol);
    memcpy(cur, bands, sizeof(double) * bvol);
    for (int a = 0; a < ndim; ++a) m[a] /= 2;
  }
  memcpy(pyr + pyr_approx_offset(ndim, n, J), cur, sizeof(double) * vol3(m));
  free(cur); free(bands); free(tmp);
  return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Training image state (Algorithm 1, line 2: DWT of the TI at level J).      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int ndim, F, J, s;
  int32_t n[3];    /* cropped fine dims (multiples of s) */
  int32_t nc[3];   /* level-J dims n / s */
  uint8_t* ti;     /* cropped TI codes */
  int64_t* cA_ind; /* [F][nc]: cA_J of the indicator image of each facies */
  int64_t* cA_code;/* [nc]: cA_J of the code image */
  int64_t* pyr;    /* full J-level pyramid of the code image (orc_dwt layout) */
} orc_ti;

static int64_t vol32(const int32_t n[3]) { return (int64_t)n[0] * n[1] * n[2]; }

void orc_ti_free(orc_ti* t) {
  if (!t) return;
  free(t->ti);
  free(t->cA_ind);
  free(t->cA_code);
  free(t->pyr);
  free(t);
}

/* Crop the TI to multiples of s = 2^J (Sec. 4.3: the level-j size is N/2^j),
 * then take the J-level DWT of the code image and of each facies indicator. */
orc_ti* orc_ti_prepare(const uint8_t* ti, int ndim, const int32_t dims[3], int F, int J) {
  if (ndim < 2 || ndim > 3 || F < 2 || F > 8 || J < 0 || J > 6) return NULL;
  orc_ti* t = (orc_ti*)calloc(1, sizeof(orc_ti));
  if (!t) return NULL;
  t->ndim = ndim;
  t->F = F;
  t->J = J;
  t->s = 1 << J;
  for (int a = 0; a < 3; ++a) {
    int32_t d = (a < ndim) ? dims[a] : 1;
    int32_t s = (a < ndim) ? t->s : 1;
    t->n[a] = (d / s) * s;
    t->nc[a] = d / s;
    if (t->nc[a] <= 0) {
      free(t);
      return NULL;
    }
  }
  int64_t nv = vol32(t->n), ncv = vol32(t->nc);
  t->ti = (uint8_t*)malloc(nv);
  t->cA_ind = (int64_t*)malloc(sizeof(int64_t) * ncv * F);
  t->cA_code = (int64_t*)malloc(sizeof(int64_t) * ncv);
  t->pyr = (int64_t*)malloc(sizeof(int64_t) * nv);
  int64_t* img = (int64_t*)malloc(sizeof(int64_t) * nv);
  int64_t* pyr = (int64_t*)malloc(sizeof(int64_t) * nv);
  if (!t->ti || !t->cA_ind || !t->cA_code || !t->pyr || !img || !pyr) {
    free(img); free(pyr);
    orc_ti_free(t);
    return NULL;
  }
  int32_t fd0 = dims[0], fd1 = ndim > 1 ? dims[1] : 1;
  for (int32_t z = 0; z < t->n[2]; ++z)
    for (int32_t y = 0; y < t->n[1]; ++y)
      for (int32_t x = 0; x < t->n[0]; ++x) {
        uint8_t v = ti[x + (int64_t)fd0 * (y + (int64_t)fd1 * z)];
        if (v >= F) {
          free(img); free(pyr);
          orc_ti_free(t);
          return NULL;
        }
        t->ti[x + (int64_t)t->n[0] * (y + (int64_t)t->n[1] * z)] = v;
      }
  int64_t aoff = pyr_approx_offset(ndim, (int64_t[3]){t->n[0], t->n[1], t->n[2]}, J);
  for (int f = 0; f < F; ++f) {
    for (int64_t i = 0; i < nv; ++i) img[i] = (t->ti[i] == f) ? 1 : 0;
    orc_dwt(img, ndim, t->n, J, pyr);
    memcpy(t->cA_ind + f * ncv, pyr + aoff, sizeof(int64_t) * ncv);
  }
  for (int64_t i = 0; i < nv; ++i) img[i] = t->ti[i];
  orc_dwt(img, ndim, t->n, J, t->pyr);
  memcpy(t->cA_code, t->pyr + aoff, sizeof(int64_t) * ncv);
  free(img);
  free(pyr);
  return t;
}

/* info[0..5] = ndim, F, J, s, ; n[3] -> info[4..6]; nc[3] -> info[7..9] */
void orc_ti_info(const orc_ti* t, int32_t info[10]) {
  info[0] = t->ndim; info[1] = t->F; info[2] = t->J; info[3] = t->s;
  for (int a = 0; a < 3; ++a) {
    info[4 + a] = t->n[a];
    info[7 + a] = t->nc[a];
  }
}

void orc_ti_get(const orc_ti* t, int64_t* cA_ind, int64_t* cA_code, int64_t* pyr,
                uint8_t* ti_cropped) {
  int64_t nv = vol32(t->n), ncv = vol32(t->nc);
  if (cA_ind) memcpy(cA_ind, t->cA_ind, sizeof(int64_t) * ncv * t->F);
  if (cA_code) memcpy(cA_code, t->cA_code, sizeof(int64_t) * ncv);
  if (pyr) memcpy(pyr, t->pyr, sizeof(int64_t) * nv);
  if (ti_cropped) memcpy(ti_cropped, t->ti, nv);
}

/* ------------------------------------------------------------------------ */
/* Best-match search for one data event (Algorithm 1, lines 8-12; Sec. 4.3, */
/* Eq. CCW; Sec. 4.4 conditional check).                                     */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t mis;
  int64_t score;
  int32_t idx;
} orc_cand;

/* 1 when a ranks before b: fewer mismatches, then higher score, then lower
 * index. */
static int cand_before(const orc_cand* a, const orc_cand* b) {
  if (a->mis != b->mis) return a->mis < b->mis;
  if (a->score != b->score) return a->score > b->score;
  return a->idx < b->idx;
}

/* Candidate grid of a template of edge T (fine cells): the level-J origins
 * x with x + T/s <= nc along every axis. */
static int cand_dims(const orc_ti* t, int T, int32_t cd[3]) {
  if (T <= 0 || T % t->s != 0) return ORC_EINVAL;
  int tj = T / t->s;
  for (int a = 0; a < 3; ++a) {
    cd[a] = (a < t->ndim) ? t->nc[a] - tj + 1 : 1;
    if (cd[a] <= 0) return ORC_EINVAL;
  }
  return ORC_OK;
}

int64_t orc_num_candidates(const orc_ti* t, int T) {
  int32_t cd[3];
  if (cand_dims(t, T, cd) != ORC_OK) return -1;
  return vol32(cd);
}

/*
 * de[T^d]: the data event (facies code, or 255 where unknown); it already
 * holds the hard data of the window. hd[T^d]: the hard data of the window
 * (255 where none); may be NULL. Writes the first min(K, P_c) candidates in
 * rank order and the picked candidate. scores/mis, when non-NULL, receive
 * the full CCW map and mismatch map over all P_c candidates.
 * Returns the number of ranked candidates written (0 for an empty data
 * event, whose pick is uniform), or a negative error.
 */
static int search_core(const orc_ti* t, int T, const uint8_t* de, const uint8_t* hd,
                       const int32_t* vhd, int n_vhd, int K, int score_mode, uint64_t seed,
                       uint32_t r, uint32_t p, int64_t* scores, int32_t* mis,
                       int32_t* topk_idx, int64_t* topk_score, int32_t* topk_mis,
                       int32_t* pick_out) {
  int32_t cd[3];
  if (cand_dims(t, T, cd) != ORC_OK || K < 1 || (score_mode != 0 && score_mode != 1))
    return ORC_EINVAL;
  const int d = t->ndim, s = t->s, J = t->J, F = t->F;
  const int tj = T / s;
  const int32_t tw[3] = {T, d > 1 ? T : 1, d > 2 ? T : 1};
  const int32_t tc[3] = {tj, d > 1 ? tj : 1, d > 2 ? tj : 1};
  const int64_t tv = vol32(tw), tcv = vol32(tc), P = vol32(cd);

  /* Algorithm 1, line 8: the overlapping region = the known cells */
  int64_t known = 0;
  for (int64_t q = 0; q < tv; ++q) {
    if (de[q] != UNKNOWN && de[q] >= F) return ORC_EINVAL;
    if (de[q] != UNKNOWN) ++known;
  }
  uint32_t u = draw_u32(seed, r, p, 0u);
  if (known == 0) {
    /* Algorithm 1, lines 5-6: nothing simulated here, draw a TI patch */
    *pick_out = (int32_t)scale_u32(u, P);
    if (scores)
      for (int64_t c = 0; c < P; ++c) scores[c] = 0;
    if (mis)
      for (int64_t c = 0; c < P; ++c) mis[c] = 0;
    return 0;
  }

  /* Algorithm 1, line 9: DWT of the OR at level J, one image per channel */
  int nch = (score_mode == 0) ? F : 1;
  int64_t* img = (int64_t*)malloc(sizeof(int64_t) * tv);
  int64_t* pyr = (int64_t*)malloc(sizeof(int64_t) * tv);
  int64_t* cor = (int64_t*)malloc(sizeof(int64_t) * tcv * nch);
  orc_cand* best = (orc_cand*)malloc(sizeof(orc_cand) * K);
  if (!img || !pyr || !cor || !best) {
    free(img); free(pyr); free(cor); free(best);
    return ORC_ENOMEM;
  }
  int64_t aoff = pyr_approx_offset(d, (int64_t[3]){tw[0], tw[1], tw[2]}, J);
  for (int ch = 0; ch < nch; ++ch) {
    for (int64_t q = 0; q < tv; ++q) {
      if (de[q] == UNKNOWN) img[q] = 0;
      else img[q] = (score_mode == 0) ? (de[q] == ch ? 1 : 0) : (int64_t)de[q];
    }
    orc_dwt(img, d, tw, J, pyr);
    memcpy(cor + ch * tcv, pyr + aoff, sizeof(int64_t) * tcv);
  }

  /* Algorithm 1, line 10: CCW(x) = sum_u cA_TI(x + u) * cA_OR(u), summed over
   * the channels; lines 11-12 and Sec. 4.4: rank, keep K, draw one. */
  const int64_t ncv = vol32(t->nc);
  const int64_t* cA = (score_mode == 0) ? t->cA_ind : t->cA_code;
  int nbest = 0;
  const int kk = (int)((K < P) ? K : P);
  for (int32_t cz = 0; cz < cd[2]; ++cz)
    for (int32_t cy = 0; cy < cd[1]; ++cy)
      for (int32_t cx = 0; cx < cd[0]; ++cx) {
        int64_t c = cx + (int64_t)cd[0] * (cy + (int64_t)cd[1] * cz);
        int64_t sc = 0;
        for (int ch = 0; ch < nch; ++ch) {
          const int64_t* a = cA + ch * ncv;
          const int64_t* w = cor + ch * tcv;
          for (int32_t uz = 0; uz < tc[2]; ++uz)
            for (int32_t uy = 0; uy < tc[1]; ++uy)
              for (int32_t ux = 0; ux < tc[0]; ++ux) {
                int64_t wv = w[ux + (int64_t)tc[0] * (uy + (int64_t)tc[1] * uz)];
                if (wv == 0) continue;
                sc += wv * a[(cx + ux) + (int64_t)t->nc[0] *
                                             ((cy + uy) + (int64_t)t->nc[1] * (cz + uz))];
              }
        }
        int32_t mm = 0;
        if (hd) {
          for (int32_t qz = 0; qz < tw[2]; ++qz)
            for (int32_t qy = 0; qy < tw[1]; ++qy)
              for (int32_t qx = 0; qx < tw[0]; ++qx) {
                uint8_t h = hd[qx + (int64_t)tw[0] * (qy + (int64_t)tw[1] * qz)];
                if (h == UNKNOWN) continue;
                int64_t fx = (int64_t)s * cx + qx, fy = (int64_t)s * cy + qy,
                        fz = (int64_t)(d > 2 ? s : 1) * cz + qz;
                if (t->ti[fx + (int64_t)t->n[0] * (fy + (int64_t)t->n[1] * fz)] != h) ++mm;
              }
        }
        /* hard data of the virtual template: a datum whose TI position lies
         * outside the TI cannot be honoured and counts as a mismatch */
        for (int v = 0; v < n_vhd; ++v) {
          const int32_t* e = vhd + 4 * v;
          int64_t fx = (int64_t)s * cx + e[0], fy = (int64_t)(d > 1 ? s : 1) * cy + e[1],
                  fz = (int64_t)(d > 2 ? s : 1) * cz + e[2];
          if (fx < 0 || fy < 0 || fz < 0 || fx >= t->n[0] || fy >= t->n[1] || fz >= t->n[2] ||
              t->ti[fx + (int64_t)t->n[0] * (fy + (int64_t)t->n[1] * fz)] != (uint8_t)e[3])
            ++mm;
        }
        if (scores) scores[c] = sc;
        if (mis) mis[c] = mm;
        /* keep the kk best in rank order (equivalent to a full sort followed
         * by taking the first kk entries, since the order is total) */
        orc_cand e = {mm, sc, (int32_t)c};
        if (nbest < kk || cand_before(&e, &best[nbest - 1])) {
          int pos = (nbest < kk) ? nbest : kk - 1;
          while (pos > 0 && cand_before(&e, &best[pos - 1])) {
            best[pos] = best[pos - 1];
            --pos;
          }
          best[pos] = e;
          if (nbest < kk) ++nbest;
        }
      }
  for (int i = 0; i < nbest; ++i) {
    topk_idx[i] = best[i].idx;
    topk_score[i] = best[i].score;
    topk_mis[i] = best[i].mis;
  }
  *pick_out = best[scale_u32(u, nbest)].idx;
  free(img); free(pyr); free(cor); free(best);
  return nbest;
}

int orc_search(const orc_ti* t, int T, const uint8_t* de, const uint8_t* hd, int K,
               int score_mode, uint64_t seed, uint32_t r, uint32_t p, int64_t* scores,
               int32_t* mis, int32_t* topk_idx, int64_t* topk_score, int32_t* topk_mis,
               int32_t* pick_out) {
  return search_core(t, T, de, hd, NULL, 0, K, score_mode, seed, r, p, scores, mis, topk_idx,
                     topk_score, topk_mis, pick_out);
}

/* orc_search with the hard data of a virtual template (Sec. 4.4 reading in
 * the header): vhd is int32 [n_vhd][4] = (qx, qy, qz, code), the datum's
 * fine offset from the window origin (any sign) and its facies. */
int orc_search_virtual(const orc_ti* t, int T, const uint8_t* de, const uint8_t* hd,
                       const int32_t* vhd, int n_vhd, int K, int score_mode, uint64_t seed,
                       uint32_t r, uint32_t p, int64_t* scores, int32_t* mis,
                       int32_t* topk_idx, int64_t* topk_score, int32_t* topk_mis,
                       int32_t* pick_out) {
  if (n_vhd < 0 || (n_vhd > 0 && !vhd)) return ORC_EINVAL;
  for (int v = 0; v < n_vhd; ++v)
    if (vhd[4 * v + 3] < 0 || vhd[4 * v + 3] >= t->F) return ORC_EINVAL;
  return search_core(t, T, de, hd, vhd, n_vhd, K, score_mode, seed, r, p, scores, mis,
                     topk_idx, topk_score, topk_mis, pick_out);
}

/* All-shift candidates (the polyphase reading in the header): the search of
 * search_core over every fine origin c = (cx, cy, cz) of the cropped TI with
 * c + T <= n. The approximation of the TI window at c is computed from its
 * definition, the s^d block sums of the indicator (one-hot) or of the codes
 * (literal) starting at c + s u. */
static int allshift_core(const orc_ti* t, int T, const uint8_t* de, const uint8_t* hd,
                         const int32_t* vhd, int n_vhd, int K, int score_mode, uint64_t seed,
                         uint32_t r, uint32_t p, int64_t* scores, int32_t* mis,
                         int32_t* topk_idx, int64_t* topk_score, int32_t* topk_mis,
                         int32_t* pick_out) {
  const int d = t->ndim, s = t->s, J = t->J, F = t->F;
  if (T <= 0 || T % s != 0 || K < 1 || (score_mode != 0 && score_mode != 1)) return ORC_EINVAL;
  int32_t fd[3];
  for (int a = 0; a < 3; ++a) {
    fd[a] = (a < d) ? t->n[a] - T + 1 : 1;
    if (fd[a] <= 0) return ORC_EINVAL;
  }
  const int tj = T / s;
  const int32_t tw[3] = {T, d > 1 ? T : 1, d > 2 ? T : 1};
  const int32_t tc[3] = {tj, d > 1 ? tj : 1, d > 2 ? tj : 1};
  const int32_t sb[3] = {s, d > 1 ? s : 1, d > 2 ? s : 1};
  const int64_t tv = vol32(tw), tcv = vol32(tc), P = vol32(fd);
  int64_t known = 0;
  for (int64_t q = 0; q < tv; ++q) {
    if (de[q] != UNKNOWN && de[q] >= F) return ORC_EINVAL;
    if (de[q] != UNKNOWN) ++known;
  }
  uint32_t u = draw_u32(seed, r, p, 0u);
  if (known == 0) {
    *pick_out = (int32_t)scale_u32(u, P);
    if (scores)
      for (int64_t c = 0; c < P; ++c) scores[c] = 0;
    if (mis)
      for (int64_t c = 0; c < P; ++c) mis[c] = 0;
    return 0;
  }
  int nch = (score_mode == 0) ? F : 1;
  int64_t* img = (int64_t*)malloc(sizeof(int64_t) * tv);
  int64_t* pyr = (int64_t*)malloc(sizeof(int64_t) * tv);
  int64_t* cor = (int64_t*)malloc(sizeof(int64_t) * tcv * nch);
  orc_cand* best = (orc_cand*)malloc(sizeof(orc_cand) * K);
  if (!img || !pyr || !cor || !best) {
    free(img); free(pyr); free(cor); free(best);
    return ORC_ENOMEM;
  }
  /* the data event's level-J approximation, as in search_core */
  int64_t aoff = pyr_approx_offset(d, (int64_t[3]){tw[0], tw[1], tw[2]}, J);
  for (int ch = 0; ch < nch; ++ch) {
    for (int64_t q = 0; q < tv; ++q) {
      if (de[q] == UNKNOWN) img[q] = 0;
      else img[q] = (score_mode == 0) ? (de[q] == ch ? 1 : 0) : (int64_t)de[q];
    }
    orc_dwt(img, d, tw, J, pyr);
    memcpy(cor + ch * tcv, pyr + aoff, sizeof(int64_t) * tcv);
  }
  int nbest = 0;
  const int kk = (int)((K < P) ? K : P);
  for (int32_t cz = 0; cz < fd[2]; ++cz)
    for (int32_t cy = 0; cy < fd[1]; ++cy)
      for (int32_t cx = 0; cx < fd[0]; ++cx) {
        const int64_t c = cx + (int64_t)fd[0] * (cy + (int64_t)fd[1] * cz);
        int64_t sc = 0;
        for (int ch = 0; ch < nch; ++ch) {
          const int64_t* w = cor + ch * tcv;
          for (int32_t uz = 0; uz < tc[2]; ++uz)
            for (int32_t uy = 0; uy < tc[1]; ++uy)
              for (int32_t ux = 0; ux < tc[0]; ++ux) {
                const int64_t wv = w[ux + (int64_t)tc[0] * (uy + (int64_t)tc[1] * uz)];
                if (wv == 0) continue;
                int64_t a = 0;   /* block sum of the TI window at c, block u */
                for (int32_t bz = 0; bz < sb[2]; ++bz)
                  for (int32_t by = 0; by < sb[1]; ++by)
                    for (int32_t bx = 0; bx < sb[0]; ++bx) {
                      const int64_t fx = cx + (int64_t)s * ux + bx;
                      const int64_t fy = cy + (int64_t)sb[1] * uy + by;
                      const int64_t fz = cz + (int64_t)sb[2] * uz + bz;
                      const uint8_t v = t->ti[fx + (int64_t)t->n[0] * (fy + (int64_t)t->n[1] * fz)];
                      a += (score_mode == 0) ? (v == ch) : v;
                    }
                sc += wv * a;
              }
        }
        int32_t mm = 0;
        if (hd)
          for (int32_t qz = 0; qz < tw[2]; ++qz)
            for (int32_t qy = 0; qy < tw[1]; ++qy)
              for (int32_t qx = 0; qx < tw[0]; ++qx) {
                const uint8_t h = hd[qx + (int64_t)tw[0] * (qy + (int64_t)tw[1] * qz)];
                if (h == UNKNOWN) continue;
                if (t->ti[(cx + qx) + (int64_t)t->n[0] * ((cy + qy) + (int64_t)t->n[1] * (cz + qz))] != h)
                  ++mm;
              }
        for (int v = 0; v < n_vhd; ++v) {
          const int32_t* e = vhd + 4 * v;
          const int64_t fx = (int64_t)cx + e[0], fy = (int64_t)cy + e[1], fz = (int64_t)cz + e[2];
          if (fx < 0 || fy < 0 || fz < 0 || fx >= t->n[0] || fy >= t->n[1] || fz >= t->n[2] ||
              t->ti[fx + (int64_t)t->n[0] * (fy + (int64_t)t->n[1] * fz)] != (uint8_t)e[3])
            ++mm;
        }
        if (scores) scores[c] = sc;
        if (mis) mis[c] = mm;
        orc_cand e = {mm, sc, (int32_t)c};
        if (nbest < kk || cand_before(&e, &best[nbest - 1])) {
          int pos = (nbest < kk) ? nbest : kk - 1;
          while (pos > 0 && cand_before(&e, &best[pos - 1])) {
            best[pos] = best[pos - 1];
            --pos;
          }
          best[pos] = e;
          if (nbest < kk) ++nbest;
        }
      }
  for (int i = 0; i < nbest; ++i) {
    topk_idx[i] = best[i].idx;
    topk_score[i] = best[i].score;
    topk_mis[i] = best[i].mis;
  }
  *pick_out = best[scale_u32(u, nbest)].idx;
  free(img); free(pyr); free(cor); free(best);
  return nbest;
}

/* Number of all-shift candidates of a template of edge T, or -1. */
int64_t orc_num_candidates_allshift(const orc_ti* t, int T) {
  if (T <= 0 || T % t->s != 0) return -1;
  int64_t P = 1;
  for (int a = 0; a < t->ndim; ++a) {
    if (t->n[a] - T + 1 <= 0) return -1;
    P *= t->n[a] - T + 1;
  }
  return P;
}

/* orc_search_virtual over the all-shift candidates (vhd may be NULL). */
int orc_search_allshift(const orc_ti* t, int T, const uint8_t* de, const uint8_t* hd,
                        const int32_t* vhd, int n_vhd, int K, int score_mode, uint64_t seed,
                        uint32_t r, uint32_t p, int64_t* scores, int32_t* mis,
                        int32_t* topk_idx, int64_t* topk_score, int32_t* topk_mis,
                        int32_t* pick_out) {
  if (n_vhd < 0 || (n_vhd > 0 && !vhd)) return ORC_EINVAL;
  for (int v = 0; v < n_vhd; ++v)
    if (vhd[4 * v + 3] < 0 || vhd[4 * v + 3] >= t->F) return ORC_EINVAL;
  return allshift_core(t, T, de, hd, vhd, n_vhd, K, score_mode, seed, r, p, scores, mis,
                       topk_idx, topk_score, topk_mis, pick_out);
}

/* Minimum-error boundary cut of image quilting (Efros and Freeman, the IQ
 * method of Sec. 2) through an overlap strip of `rows` x `cols` cells with
 * 0/1 costs err[y * cols + x]: the cumulative cost
 *   E(0, x) = err(0, x),  E(y, x) = err(y, x) + min_{|x' - x| <= 1} E(y - 1, x'),
 * then the path traced back from the cheapest cell of the last row, each
 * step to the cheapest of the (up to) three cells above; ties go to the
 * lower column. cut[y] = the path's column in row y. */
int orc_min_cut(const uint8_t* err, int rows, int cols, int32_t* cut) {
  if (rows < 1 || cols < 1 || !err || !cut) return ORC_EINVAL;
  int64_t* E = (int64_t*)malloc(sizeof(int64_t) * rows * cols);
  if (!E) return ORC_ENOMEM;
  for (int x = 0; x < cols; ++x) E[x] = err[x];
  for (int y = 1; y < rows; ++y)
    for (int x = 0; x < cols; ++x) {
      int64_t m = E[(y - 1) * cols + x];
      if (x > 0 && E[(y - 1) * cols + x - 1] < m) m = E[(y - 1) * cols + x - 1];
      if (x + 1 < cols && E[(y - 1) * cols + x + 1] < m) m = E[(y - 1) * cols + x + 1];
      E[y * cols + x] = err[y * cols + x] + m;
    }
  int c = 0;
  for (int x = 1; x < cols; ++x)
    if (E[(rows - 1) * cols + x] < E[(rows - 1) * cols + c]) c = x;
  cut[rows - 1] = c;
  for (int y = rows - 2; y >= 0; --y) {
    int lo = c > 0 ? c - 1 : 0, hi = c + 1 < cols ? c + 1 : cols - 1, b = lo;
    for (int x = lo + 1; x <= hi; ++x)
      if (E[y * cols + x] < E[y * cols + b]) b = x;
    c = b;
    cut[y] = c;
  }
  free(E);
  return ORC_OK;
}

/* Algorithm 1, line 13: Inverse-DWT of the selected pattern. The pattern's
 * own pyramid is cut from the TI's code pyramid (approximation at the
 * candidate's level-J origin, level-j details at that origin times 2^(J-j))
 * and synthesised back to T^d fine cells. */
int orc_reconstruct(const orc_ti* t, int T, int32_t pick, uint8_t* pattern) {
  int32_t cd[3];
  if (cand_dims(t, T, cd) != ORC_OK) return ORC_EINVAL;
  if (pick < 0 || pick >= vol32(cd)) return ORC_EINVAL;
  const int d = t->ndim, J = t->J, s = t->s;
  const int32_t tw[3] = {T, d > 1 ? T : 1, d > 2 ? T : 1};
  const int64_t tv = vol32(tw);
  const int64_t nfull[3] = {t->n[0], t->n[1], t->n[2]};
  const int64_t npat[3] = {tw[0], tw[1], tw[2]};
  int32_t pc[3] = {pick % cd[0], (pick / cd[0]) % cd[1], pick / (cd[0] * cd[1])};
  int64_t* ppyr = (int64_t*)malloc(sizeof(int64_t) * tv);
  int64_t* x = (int64_t*)malloc(sizeof(int64_t) * tv);
  if (!ppyr || !x) {
    free(ppyr); free(x);
    return ORC_ENOMEM;
  }
  (void)s;
  for (int j = 1; j <= J + 1; ++j) {
    /* j <= J: detail bands of level j; j == J + 1: the approximation cA_J */
    int lev = (j <= J) ? j : J;
    int nbands = (j <= J) ? (1 << d) - 1 : 1;
    int64_t sc = (int64_t)1 << (J - lev);
    int64_t fm[3], pm[3], org[3];
    for (int a = 0; a < 3; ++a) {
      fm[a] = (a < d) ? (nfull[a] >> lev) : 1;
      pm[a] = (a < d) ? (npat[a] >> lev) : 1;
      org[a] = (a < d) ? pc[a] * sc : 0;
    }
    for (int b = 1; b <= nbands; ++b) {
      int64_t fo = (j <= J) ? pyr_band_offset(d, nfull, j, b) : pyr_approx_offset(d, nfull, J);
      int64_t po = (j <= J) ? pyr_band_offset(d, npat, j, b) : pyr_approx_offset(d, npat, J);
      for (int64_t z = 0; z < pm[2]; ++z)
        for (int64_t y = 0; y < pm[1]; ++y)
          for (int64_t xx = 0; xx < pm[0]; ++xx)
            ppyr[po + xx + pm[0] * (y + pm[1] * z)] =
                t->pyr[fo + (org[0] + xx) + fm[0] * ((org[1] + y) + fm[1] * (org[2] + z))];
    }
  }
  int rc = orc_idwt(ppyr, d, tw, J, x);
  if (rc == ORC_OK)
    for (int64_t q = 0; q < tv; ++q) pattern[q] = (uint8_t)x[q];
  free(ppyr); free(x);
  return rc;
}

/* ------------------------------------------------------------------------ */
/* Raster-path simulation of one realization (Algorithm 1; Sec. 4.1 lattice, */
/* Sec. 4.4 conditioning).                                                   */
/* ------------------------------------------------------------------------ */

/* Lattice of Sec. 4.1: patches of edge T stepping by S = T - O, n_a patches
 * along axis a so that the padded extent T + (n_a - 1) S covers the grid. */
int orc_lattice(int ndim, const int32_t grid[3], int T, int O, int32_t n_out[3],
                int32_t gp_out[3]) {
  int S = T - O;
  if (S <= 0) return ORC_EINVAL;
  for (int a = 0; a < 3; ++a) {
    if (a >= ndim) {
      n_out[a] = 1;
      gp_out[a] = 1;
      continue;
    }
    int32_t g = grid[a];
    int32_t extra = g > T ? g - T : 0;
    n_out[a] = 1 + (extra + S - 1) / S;
    gp_out[a] = T + (n_out[a] - 1) * S;
  }
  return ORC_OK;
}

/* Path orientation of realization r: bit a set = the raster runs backwards
 * along axis a (Algorithm 1, line 3, "Randomize(origin, direction)"). */
uint32_t orc_path_flips(int ndim, uint64_t seed, uint32_t r, int path_random) {
  if (!path_random) return 0;
  return draw_u32(seed, r, 0u, 1u) & ((1u << ndim) - 1u);
}

/*
 * Simulates realization r of a grid of dims `grid`. `hd_cells` is int32
 * [n_hd][ndim] (x, y, z), `hd_vals` u8 [n_hd]; when two hard data share a
 * cell the smaller code is kept. Writes the grid to `out` (cells never
 * simulated, possible only with max_patches, are 255). `log`, when non-NULL,
 * receives per patch (in path order) the int32 record
 *   {pick, score of pick, mismatches of pick, flags, topk[0..K-1]}
 * with flags bit0 = uniform pick (empty data event), bit1 = patch done, and
 * unused topk slots = -1. Stops after max_patches patches when >= 0.
 * vt_ext (0..T) grows the virtual template of the non-causal conditioning;
 * cut = 1 pastes through the minimum-error boundary cuts (2D only);
 * all_shift = 1 searches the all-shift candidates (pick and log indices are
 * then fine-grid indices). All follow the readings in the header;
 * orc_simulate is vt_ext = cut = all_shift = 0.
 */
int orc_simulate_ext(const orc_ti* t, const int32_t grid[3], int T, int O, int K,
                     int score_mode, int path_random, int vt_ext, int cut, int all_shift,
                     int n_hd, const int32_t* hd_cells, const uint8_t* hd_vals, uint64_t seed,
                     uint32_t r, int64_t max_patches, uint8_t* out, int32_t* log) {
  const int d = t->ndim;
  if (T % t->s != 0 || O % t->s != 0 || O < 0 || T < 2 * O || K < 1) return ORC_EINVAL;
  if (vt_ext < 0 || vt_ext > T || (cut != 0 && cut != 1) || (cut && d != 2)) return ORC_EINVAL;
  if (all_shift != 0 && all_shift != 1) return ORC_EINVAL;
  if (all_shift && orc_num_candidates_allshift(t, T) < 0) return ORC_EINVAL;
  int32_t np[3], gp[3], cd[3];
  if (orc_lattice(d, grid, T, O, np, gp) != ORC_OK) return ORC_EINVAL;
  if (cand_dims(t, T, cd) != ORC_OK) return ORC_EINVAL;
  const int S = T - O;
  const int32_t g3[3] = {grid[0], d > 1 ? grid[1] : 1, d > 2 ? grid[2] : 1};
  const int32_t tw[3] = {T, d > 1 ? T : 1, d > 2 ? T : 1};
  const int64_t tv = vol32(tw), gpv = vol32(gp);
  const uint32_t flips = orc_path_flips(d, seed, r, path_random);
  int32_t off[3];
  for (int a = 0; a < 3; ++a) off[a] = (flips >> a & 1u) ? gp[a] - g3[a] : 0;

  uint8_t* sg = (uint8_t*)malloc(gpv);
  uint8_t* hdo = (uint8_t*)malloc(gpv);
  uint8_t* de = (uint8_t*)malloc(tv);
  uint8_t* hw = (uint8_t*)malloc(tv);
  uint8_t* pat = (uint8_t*)malloc(tv);
  int32_t* ti_idx = (int32_t*)malloc(sizeof(int32_t) * K);
  int64_t* ti_sc = (int64_t*)malloc(sizeof(int64_t) * K);
  int32_t* ti_mm = (int32_t*)malloc(sizeof(int32_t) * K);
  int64_t* scores = NULL;
  int32_t* mism = NULL;
  /* the virtual template: the window grown by vt_ext cells along the
   * forward direction of every axis of the path */
  const int32_t gw[3] = {T + vt_ext, d > 1 ? T + vt_ext : 1, d > 2 ? T + vt_ext : 1};
  const int64_t n_vmax = vt_ext ? vol32(gw) - tv : 0;
  int32_t* vhd = (int32_t*)malloc(sizeof(int32_t) * 4 * (n_vmax > 0 ? n_vmax : 1));
  uint8_t* errv = (uint8_t*)malloc((size_t)T * (O > 0 ? O : 1));
  uint8_t* errh = (uint8_t*)malloc((size_t)T * (O > 0 ? O : 1));
  int32_t* cutv = (int32_t*)malloc(sizeof(int32_t) * T);
  int32_t* cuth = (int32_t*)malloc(sizeof(int32_t) * T);
  int rc = ORC_OK;
  if (!sg || !hdo || !de || !hw || !pat || !ti_idx || !ti_sc || !ti_mm || !vhd || !errv ||
      !errh || !cutv || !cuth) {
    rc = ORC_ENOMEM;
    goto done;
  }
  memset(sg, UNKNOWN, gpv);
  memset(hdo, UNKNOWN, gpv);
  for (int i = 0; i < n_hd; ++i) {
    int32_t c[3] = {0, 0, 0};
    for (int a = 0; a < d; ++a) c[a] = hd_cells[i * d + a];
    for (int a = 0; a < 3; ++a)
      if (c[a] < 0 || c[a] >= g3[a]) {
        rc = ORC_EINVAL;
        goto done;
      }
    if (hd_vals[i] >= t->F) {
      rc = ORC_EINVAL;
      goto done;
    }
    int64_t cell = (c[0] + off[0]) + (int64_t)gp[0] * ((c[1] + off[1]) + (int64_t)gp[1] * (c[2] + off[2]));
    if (hd_vals[i] < hdo[cell]) hdo[cell] = hd_vals[i];
  }

  const int64_t npatch = (int64_t)np[0] * np[1] * np[2];
  const int stride = 4 + K;
  if (log)
    for (int64_t i = 0; i < npatch * stride; ++i) log[i] = (i % stride == 3) ? 0 : -1;
  for (int64_t p = 0; p < npatch; ++p) {
    if (max_patches >= 0 && p >= max_patches) break;
    int32_t ip[3] = {(int32_t)(p % np[0]), (int32_t)((p / np[0]) % np[1]),
                     (int32_t)(p / ((int64_t)np[0] * np[1]))};
    int32_t o[3];
    for (int a = 0; a < 3; ++a)
      o[a] = (flips >> a & 1u) ? gp[a] - tw[a] - S * ip[a] : S * ip[a];
    if (d < 3) o[2] = 0;
    if (d < 2) o[1] = 0;
    /* Algorithm 1, line 8: the data event of the window, hard data first */
    for (int32_t qz = 0; qz < tw[2]; ++qz)
      for (int32_t qy = 0; qy < tw[1]; ++qy)
        for (int32_t qx = 0; qx < tw[0]; ++qx) {
          int64_t q = qx + (int64_t)tw[0] * (qy + (int64_t)tw[1] * qz);
          int64_t cell = (o[0] + qx) + (int64_t)gp[0] * ((o[1] + qy) + (int64_t)gp[1] * (o[2] + qz));
          hw[q] = hdo[cell];
          de[q] = (hdo[cell] != UNKNOWN) ? hdo[cell] : sg[cell];
        }
    /* the hard data of the virtual template outside the template; path
     * frame (x', y', z') = window offsets mirrored along flipped axes */
    int n_vhd = 0;
    for (int32_t vz = 0; vz < gw[2]; ++vz)
      for (int32_t vy = 0; vy < gw[1]; ++vy)
        for (int32_t vx = 0; vx < gw[0]; ++vx) {
          if (vx < tw[0] && vy < tw[1] && vz < tw[2]) continue;   /* template cell */
          const int32_t v3[3] = {vx, vy, vz};
          int32_t q3[3];
          int inside = 1;
          for (int a = 0; a < 3; ++a) {
            q3[a] = (flips >> a & 1u) ? tw[a] - 1 - v3[a] : v3[a];
            const int64_t gc = (int64_t)o[a] + q3[a];
            if (gc < 0 || gc >= gp[a]) inside = 0;
          }
          if (!inside) continue;
          const uint8_t h =
              hdo[(o[0] + q3[0]) + (int64_t)gp[0] * ((o[1] + q3[1]) + (int64_t)gp[1] * (o[2] + q3[2]))];
          if (h == UNKNOWN) continue;
          vhd[4 * n_vhd] = q3[0];
          vhd[4 * n_vhd + 1] = q3[1];
          vhd[4 * n_vhd + 2] = q3[2];
          vhd[4 * n_vhd + 3] = h;
          ++n_vhd;
        }
    int32_t pick = -1;
    int nk = all_shift
                 ? allshift_core(t, T, de, hw, vhd, n_vhd, K, score_mode, seed, r, (uint32_t)p,
                                 scores, mism, ti_idx, ti_sc, ti_mm, &pick)
                 : search_core(t, T, de, hw, vhd, n_vhd, K, score_mode, seed, r, (uint32_t)p,
                               scores, mism, ti_idx, ti_sc, ti_mm, &pick);
    if (nk < 0) {
      rc = nk;
      goto done;
    }
    /* Algorithm 1, lines 13-14: reconstruct and paste; hard data stay. An
     * all-shift candidate's pattern is the TI crop at its fine origin. */
    if (all_shift) {
      const int32_t fd0 = t->n[0] - T + 1, fd1 = d > 1 ? t->n[1] - T + 1 : 1;
      const int32_t c3[3] = {pick % fd0, (pick / fd0) % fd1, pick / (fd0 * fd1)};
      for (int32_t qz = 0; qz < tw[2]; ++qz)
        for (int32_t qy = 0; qy < tw[1]; ++qy)
          for (int32_t qx = 0; qx < tw[0]; ++qx)
            pat[qx + (int64_t)tw[0] * (qy + (int64_t)tw[1] * qz)] =
                t->ti[(c3[0] + qx) + (int64_t)t->n[0] * ((c3[1] + qy) + (int64_t)t->n[1] * (c3[2] + qz))];
    } else {
      rc = orc_reconstruct(t, T, pick, pat);
      if (rc != ORC_OK) goto done;
    }
    if (cut && O > 0) {
      /* boundary cuts in the path frame: column cut through the left strip
       * (rows y', columns x' < O), row cut through the top strip (rows x',
       * columns y' < O); the cost of a cell is 1 where the grid already
       * holds a value that differs from the pattern */
      for (int32_t yp = 0; yp < T; ++yp)
        for (int32_t xp = 0; xp < T; ++xp) {
          if (xp >= O && yp >= O) continue;
          const int32_t qx = (flips & 1u) ? T - 1 - xp : xp;
          const int32_t qy = (flips & 2u) ? T - 1 - yp : yp;
          const uint8_t old = sg[(o[0] + qx) + (int64_t)gp[0] * (o[1] + qy)];
          const uint8_t e = (old != UNKNOWN && old != pat[qx + (int64_t)T * qy]) ? 1 : 0;
          if (xp < O) errv[yp * O + xp] = e;
          if (yp < O) errh[xp * O + yp] = e;
        }
      if ((rc = orc_min_cut(errv, T, O, cutv)) != ORC_OK ||
          (rc = orc_min_cut(errh, T, O, cuth)) != ORC_OK)
        goto done;
    }
    for (int32_t qz = 0; qz < tw[2]; ++qz)
      for (int32_t qy = 0; qy < tw[1]; ++qy)
        for (int32_t qx = 0; qx < tw[0]; ++qx) {
          int64_t q = qx + (int64_t)tw[0] * (qy + (int64_t)tw[1] * qz);
          int64_t cell = (o[0] + qx) + (int64_t)gp[0] * ((o[1] + qy) + (int64_t)gp[1] * (o[2] + qz));
          if (hw[q] != UNKNOWN) {
            sg[cell] = hw[q];
            continue;
          }
          int take = 1;
          if (cut && O > 0 && sg[cell] != UNKNOWN) {
            const int32_t xp = (flips & 1u) ? T - 1 - qx : qx;
            const int32_t yp = (flips & 2u) ? T - 1 - qy : qy;
            take = xp >= cutv[yp] && yp >= cuth[xp];
          }
          if (take) sg[cell] = pat[q];
        }
    if (log) {
      int32_t* e = log + p * stride;
      e[0] = pick;
      if (nk == 0) {
        e[1] = 0;
        e[2] = 0;
        e[3] = 1 | 2;
      } else {
        int sel = -1;
        for (int i = 0; i < nk; ++i)
          if (ti_idx[i] == pick) sel = i;
        e[1] = (int32_t)ti_sc[sel];
        e[2] = ti_mm[sel];
        e[3] = 2;
        for (int i = 0; i < nk; ++i) e[4 + i] = ti_idx[i];
      }
    }
  }
  for (int32_t z = 0; z < g3[2]; ++z)
    for (int32_t y = 0; y < g3[1]; ++y)
      for (int32_t x = 0; x < g3[0]; ++x)
        out[x + (int64_t)g3[0] * (y + (int64_t)g3[1] * z)] =
            sg[(x + off[0]) + (int64_t)gp[0] * ((y + off[1]) + (int64_t)gp[1] * (z + off[2]))];
done:
  free(sg); free(hdo); free(de); free(hw); free(pat);
  free(ti_idx); free(ti_sc); free(ti_mm); free(scores); free(mism);
  free(vhd); free(errv); free(errh); free(cutv); free(cuth);
  return rc;
}

int orc_simulate(const orc_ti* t, const int32_t grid[3], int T, int O, int K,
                 int score_mode, int path_random, int n_hd, const int32_t* hd_cells,
                 const uint8_t* hd_vals, uint64_t seed, uint32_t r, int64_t max_patches,
                 uint8_t* out, int32_t* log) {
  return orc_simulate_ext(t, grid, T, O, K, score_mode, path_random, 0, 0, 0, n_hd, hd_cells,
                          hd_vals, seed, r, max_patches, out, log);
}
