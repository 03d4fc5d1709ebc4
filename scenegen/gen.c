/*
 * Seeded synthetic scene generator shared by the oracle tests and the GPU
 * benchmark.  It produces RAW Gaussian attributes in the layout of the Kerbl
 * et al. 3DGS export (position, log-scale, unnormalised-or-unit quaternion
 * (w,x,y,z), opacity logit, DC colour coefficients, higher-band SH
 * coefficients stored channel-major [c][k]).  It contains none of the
 * method's arithmetic: decoding, paging, LOD, proxy and rendering all live on
 * either side of the boundary, never here.
 *
 * Every random number is counter based: value (seed, stream, index) is
 * SplitMix64 (Steele, Lea, Flood, "Fast splittable pseudorandom number
 * generators", OOPSLA 2014) applied twice, so any element can be regenerated
 * in isolation and OpenMP threads need no shared state.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#define SG_PI 3.14159265358979323846

static inline uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

static inline uint64_t rbits(uint64_t seed, uint64_t stream, uint64_t i) {
  return sm64(sm64(seed ^ 0x5DEECE66Dull) ^ (stream << 44) ^ i);
}

/* uniform in [0, 1) with 53 random bits */
static inline double u01(uint64_t seed, uint64_t stream, uint64_t i) {
  return (double)(rbits(seed, stream, i) >> 11) * (1.0 / 9007199254740992.0);
}

/* standard normal by Box-Muller from draws 2i and 2i+1 of the stream */
static inline double nrm(uint64_t seed, uint64_t stream, uint64_t i) {
  double a = u01(seed, stream, 2 * i), b = u01(seed, stream, 2 * i + 1);
  return sqrt(-2.0 * log(1.0 - a)) * cos(2.0 * SG_PI * b);
}

enum {
  ST_POS = 1, ST_SCALE, ST_ROT, ST_OPAC, ST_DC, ST_REST, ST_BLOB, ST_BOX,
  ST_PICK, ST_FACE, ST_SPIN
};

/* Shoemake's uniform random rotation, stored (w, x, y, z) */
static void shoemake(uint64_t seed, uint64_t g, float *q) {
  double u1 = u01(seed, ST_ROT, 3 * g), u2 = u01(seed, ST_ROT, 3 * g + 1),
         u3 = u01(seed, ST_ROT, 3 * g + 2);
  double a = sqrt(1.0 - u1), b = sqrt(u1);
  q[1] = (float)(a * sin(2 * SG_PI * u2));
  q[2] = (float)(a * cos(2 * SG_PI * u2));
  q[3] = (float)(b * sin(2 * SG_PI * u3));
  q[0] = (float)(b * cos(2 * SG_PI * u3));
}

static void colour(uint64_t seed, uint64_t g, int n_rest, double rest_sd,
                   float *f_dc, float *f_rest) {
  for (int c = 0; c < 3; ++c) f_dc[3 * g + c] = (float)u01(seed, ST_DC, 3 * g + c);
  for (int j = 0; j < 3 * n_rest; ++j)
    f_rest[(uint64_t)3 * n_rest * g + j] =
        (float)(rest_sd * nrm(seed, ST_REST, (uint64_t)3 * n_rest * g + j));
}

/*
 * Config "tiny": positions uniform in [lo, hi]^3, log-scales N(ls_mu, ls_sd),
 * uniform unit quaternions, opacity logit N(op_mu, op_sd), DC U[0,1], higher
 * bands N(0, rest_sd).
 */
void sg_uniform(int64_t n, uint64_t seed, double lo, double hi, double ls_mu,
                double ls_sd, double op_mu, double op_sd, int sh_degree,
                double rest_sd, float *pos, float *log_scale, float *rot,
                float *op_logit, float *f_dc, float *f_rest) {
  int n_rest = (sh_degree + 1) * (sh_degree + 1) - 1;
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < n; ++g) {
    for (int a = 0; a < 3; ++a) {
      pos[3 * g + a] = (float)(lo + (hi - lo) * u01(seed, ST_POS, 3 * g + a));
      log_scale[3 * g + a] = (float)(ls_mu + ls_sd * nrm(seed, ST_SCALE, 3 * g + a));
    }
    shoemake(seed, g, rot + 4 * g);
    op_logit[g] = (float)(op_mu + op_sd * nrm(seed, ST_OPAC, g));
    colour(seed, g, n_rest, rest_sd, f_dc, f_rest);
  }
}

/*
 * Config "blobs": n_blobs isotropic normal clusters of std blob_sigma whose
 * centres are uniform in [lo, hi]^3; Gaussian g belongs to blob
 * floor(g * n_blobs / n).  Other attributes as in sg_uniform.
 */
void sg_blobs(int64_t n, uint64_t seed, int n_blobs, double blob_sigma,
              double lo, double hi, double ls_mu, double ls_sd, double op_mu,
              double op_sd, int sh_degree, double rest_sd, float *pos,
              float *log_scale, float *rot, float *op_logit, float *f_dc,
              float *f_rest) {
  int n_rest = (sh_degree + 1) * (sh_degree + 1) - 1;
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < n; ++g) {
    int64_t b = (g * n_blobs) / n;
    for (int a = 0; a < 3; ++a) {
      double c = lo + (hi - lo) * u01(seed, ST_BLOB, 3 * b + a);
      pos[3 * g + a] = (float)(c + blob_sigma * nrm(seed, ST_POS, 3 * g + a));
      log_scale[3 * g + a] = (float)(ls_mu + ls_sd * nrm(seed, ST_SCALE, 3 * g + a));
    }
    shoemake(seed, g, rot + 4 * g);
    op_logit[g] = (float)(op_mu + op_sd * nrm(seed, ST_OPAC, g));
    colour(seed, g, n_rest, rest_sd, f_dc, f_rest);
  }
}

/* box b of the city: x0, y0, w (x extent), d (y extent), h (height) */
static void city_box(uint64_t seed, int64_t b, double extent, double *bx) {
  double w = 10.0 + 50.0 * u01(seed, ST_BOX, 5 * b + 2);
  double d = 10.0 + 50.0 * u01(seed, ST_BOX, 5 * b + 3);
  double h = 10.0 + 70.0 * u01(seed, ST_BOX, 5 * b + 4);
  bx[0] = (extent - w) * u01(seed, ST_BOX, 5 * b + 0);
  bx[1] = (extent - d) * u01(seed, ST_BOX, 5 * b + 1);
  bx[2] = w; bx[3] = d; bx[4] = h;
}

static void qmul(const double *a, const double *b, double *o) {
  o[0] = a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3];
  o[1] = a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2];
  o[2] = a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1];
  o[3] = a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0];
}

/*
 * Config "city": a extent x extent ground plane (world z up, z = 0) with
 * n_boxes axis-aligned boxes (footprint U[10,60] m per side, height
 * U[10,80] m).  The first floor(ground_frac * n) Gaussians lie on the
 * ground, the rest on box walls and roofs, uniform by area.  Each Gaussian is
 * flattened along the surface normal: tangent std 0.6*sqrt(area/count) times
 * exp(N(0, 0.2)), normal std one tenth of that, random spin about the normal.
 * Opacity logit N(op_mu, op_sd).  box_area_cdf is caller scratch of n_boxes
 * doubles.
 */
void sg_city(int64_t n, uint64_t seed, int n_boxes, double extent,
             double ground_frac, double op_mu, double op_sd, int sh_degree,
             double rest_sd, double *box_area_cdf, float *pos,
             float *log_scale, float *rot, float *op_logit, float *f_dc,
             float *f_rest) {
  int n_rest = (sh_degree + 1) * (sh_degree + 1) - 1;
  int64_t n_ground = (int64_t)floor(ground_frac * (double)n);
  int64_t n_surf = n - n_ground;
  double total = 0.0;
  for (int b = 0; b < n_boxes; ++b) {
    double bx[5];
    city_box(seed, b, extent, bx);
    total += 2.0 * (bx[2] + bx[3]) * bx[4] + bx[2] * bx[3];
    box_area_cdf[b] = total;
  }
  double sig_g = 0.6 * sqrt(extent * extent / (double)(n_ground > 0 ? n_ground : 1));
  double sig_s = 0.6 * sqrt(total / (double)(n_surf > 0 ? n_surf : 1));
#pragma omp parallel for schedule(static)
  for (int64_t g = 0; g < n; ++g) {
    double p[3], nrmq[4], sig;
    if (g < n_ground) {
      p[0] = extent * u01(seed, ST_POS, 3 * g);
      p[1] = extent * u01(seed, ST_POS, 3 * g + 1);
      p[2] = 0.0;
      nrmq[0] = 1; nrmq[1] = nrmq[2] = nrmq[3] = 0;   /* local z = +z */
      sig = sig_g;
    } else {
      double t = total * u01(seed, ST_PICK, g);
      int lo = 0, hi = n_boxes - 1;
      while (lo < hi) { int mid = (lo + hi) / 2; if (box_area_cdf[mid] <= t) lo = mid + 1; else hi = mid; }
      double bx[5];
      city_box(seed, lo, extent, bx);
      double w = bx[2], d = bx[3], h = bx[4];
      double areas[5] = {w * h, w * h, d * h, d * h, w * d};
      double f = (areas[0] + areas[1] + areas[2] + areas[3] + areas[4]) * u01(seed, ST_FACE, g);
      int face = 0;
      while (face < 4 && f >= areas[face]) { f -= areas[face]; ++face; }
      double a = u01(seed, ST_POS, 3 * g), c = u01(seed, ST_POS, 3 * g + 1);
      const double s = 0.70710678118654752;
      switch (face) {
        case 0: p[0] = bx[0] + a * w; p[1] = bx[1];     p[2] = c * h;                 /* -y wall */
                nrmq[0] = s; nrmq[1] = s; nrmq[2] = 0; nrmq[3] = 0; break;
        case 1: p[0] = bx[0] + a * w; p[1] = bx[1] + d; p[2] = c * h;                 /* +y wall */
                nrmq[0] = s; nrmq[1] = -s; nrmq[2] = 0; nrmq[3] = 0; break;
        case 2: p[0] = bx[0];     p[1] = bx[1] + a * d; p[2] = c * h;                 /* -x wall */
                nrmq[0] = s; nrmq[1] = 0; nrmq[2] = -s; nrmq[3] = 0; break;
        case 3: p[0] = bx[0] + w; p[1] = bx[1] + a * d; p[2] = c * h;                 /* +x wall */
                nrmq[0] = s; nrmq[1] = 0; nrmq[2] = s; nrmq[3] = 0; break;
        default: p[0] = bx[0] + a * w; p[1] = bx[1] + c * d; p[2] = h;                /* roof */
                nrmq[0] = 1; nrmq[1] = nrmq[2] = nrmq[3] = 0; break;
      }
      sig = sig_s;
    }
    double ang = 2.0 * SG_PI * u01(seed, ST_SPIN, g);
    double spin[4] = {cos(0.5 * ang), 0, 0, sin(0.5 * ang)}, q[4];
    qmul(nrmq, spin, q);
    for (int k = 0; k < 3; ++k) pos[3 * g + k] = (float)p[k];
    for (int k = 0; k < 4; ++k) rot[4 * g + k] = (float)q[k];
    log_scale[3 * g + 0] = (float)(log(sig) + 0.2 * nrm(seed, ST_SCALE, 3 * g + 0));
    log_scale[3 * g + 1] = (float)(log(sig) + 0.2 * nrm(seed, ST_SCALE, 3 * g + 1));
    log_scale[3 * g + 2] = (float)(log(0.1 * sig) + 0.2 * nrm(seed, ST_SCALE, 3 * g + 2));
    op_logit[g] = (float)(op_mu + op_sd * nrm(seed, ST_OPAC, g));
    colour(seed, g, n_rest, rest_sd, f_dc, f_rest);
  }
}

/* the city's boxes, for building camera paths that avoid them */
void sg_city_boxes(uint64_t seed, int n_boxes, double extent, double *out5) {
  for (int b = 0; b < n_boxes; ++b) city_box(seed, b, extent, out5 + 5 * b);
}

/* uniform [0,1) draws of an arbitrary stream, for camera-path construction */
void sg_u01(uint64_t seed, uint64_t stream, int64_t n, double *out) {
  for (int64_t i = 0; i < n; ++i) out[i] = u01(seed, stream + 64, i);
}
