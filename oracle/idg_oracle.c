/*
 * idg_oracle.c -- plain FP64 CPU oracle for image-domain gridding (IDG).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the GPU library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg and reference arm of the
 * benchmark load it.  It shares no code, header, table or helper with the
 * CUDA library, and the library never calls it.
 *
 * Everything here is double precision (the paper fixes no precision for the
 * reference; Section 4.1 compares against an FP64 direct transform).
 *
 * Conventions, each tied to the paper:
 *   - Visibility k of baseline b=(p,q), timestep t, channel ch is a 2x2
 *     complex Jones matrix [XX XY; YX YY] stored as 4 complex numbers.
 *   - u,v,w in wavelengths: uvw_metres * f / c                  (Section 2.1)
 *   - Grid pixel spacing du = 1/FOV; pixel coordinate of u is
 *     xi = u*FOV + N/2, the grid is [pol][y][x] with x <-> u.
 *   - A subgrid is L x L pixels with corner (x0,y0); its centre is
 *     u0 = (x0 + L/2 - N/2)/FOV                                  (Section 2.2)
 *   - Subgrid image pixel (i,j) sits at l_i=(i-L/2)FOV/L, m_j=(j-L/2)FOV/L,
 *     n'_{ij} = sqrt(1-l^2-m^2) - 1                              (Eq. 1, Eq. 7)
 *   - Gridder (Eq. 10, step 2a of Section 2.5):
 *       X(i,j) = T_i T_j sum_g A_p,g^H [ sum_{k in g} V_k e^{+2 pi i phi_k} ] A_q,g
 *       phi_k = (u_k-u0) l_i + (v_k-v0) m_j + (w_k-w0) n'_{ij},
 *     w0 = 0, or with w layers the subgrid's layer w0 = (2k+1) w_max
 *     (Section 2.4), where g runs over the A-term intervals the subgrid covers
 *     (Section 3.3: the A-term is applied after the sum over visibilities
 *     that share it).
 *   - w layers (Section 2.4 and its footnote): a timestep row (b, t) whose w
 *     is negative is gridded as its mirror, the visibility V^H of baseline
 *     (q, p) at (-u, -v, -w), since V(u,v,w) = V(-u,-v,-w)^H; so every
 *     gridded w >= 0 and the layers are {w_max, 3 w_max, 5 w_max, ...}.  The
 *     degridder predicts the mirror and returns its conjugate transpose.
 *   - Subgrid FFT (step 2b), unnormalised, centred:
 *       Vhat(x,y) = sum_{ij} X(i,j) e^{-2 pi i [(x-L/2)(i-L/2)+(y-L/2)(j-L/2)]/L}
 *   - Adder (step 2c, Eq. 6): G[pol][y0+y][x0+x] += Vhat(x,y)
 *   - Degridder (Section 2.5 prediction, Eq. 13) is the exact adjoint:
 *       splitter Yhat(x,y) = G[..][y0+y][x0+x]; unnormalised inverse DFT with
 *       the + sign; Z = T_i T_j A_p Y A_q^H; V_k = sum_ij Z e^{-2 pi i phi_k}.
 *     (Readings: A^H/A in place of A^{-1}/A, and the taper multiplied rather
 *     than divided in the degridder, make the pair exact adjoints.)
 *   - Taper (Section 4.2): Kaiser-Bessel T(l) = I0(beta sqrt(1-x^2))/I0(beta),
 *     x = 2l/FOV, separable in l and m.
 *   - A-terms: per station per interval, sampled on nodes x nodes points over
 *     [-FOV/2, FOV/2]^2 and interpolated bilinearly to the subgrid pixels.
 *
 * The partitioner follows Section 3.1 (subtables of the time x channel table
 * of one baseline, checked by their corners); the exact reading of the
 * fit-with-margin rule and of the time extension is documented at oracle_plan().
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_SPEED_OF_LIGHT 299792458.0
#define OR_PI 3.14159265358979323846

/* status codes (same numeric meaning as the library's, chosen independently) */
enum {
  OR_OK = 0,
  OR_ERR_INVALID = 1,
  OR_ERR_UNSORTED_FREQ = 2,
  OR_ERR_OUT_OF_GRID = 3,
  OR_ERR_W_TOO_LARGE = 4,
  OR_ERR_CAPACITY = 9
};

/* planner flags */
#define OR_FLAG_DROP 1
#define OR_FLAG_SPLIT_INTERVALS 2
#define OR_FLAG_W_LAYERS 4

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* coordinates                                                          */
/* ------------------------------------------------------------------ */

/* pixel coordinate along u (axis 0) or v (axis 1): ((sgn*uvw*f)/c)*FOV + N/2,
 * sgn = -1 for a mirrored row (w layers), else +1 */
static double or_pix(const double* uvw, int n_t, int b, int t, int axis, double sgn,
                     double f, double fov, int N) {
  double u_m = sgn * uvw[((size_t)b * n_t + t) * 3 + axis];
  double u_l = (u_m * f) / OR_SPEED_OF_LIGHT;
  return u_l * fov + (double)(N / 2);
}

static double or_wavelengths(const double* uvw, int n_t, int b, int t, int axis, double sgn, double f) {
  return (sgn * uvw[((size_t)b * n_t + t) * 3 + axis] * f) / OR_SPEED_OF_LIGHT;
}

/* conjugate transpose of a 2x2 visibility, the mirror's value V^H */
static void or_vis_herm(const double complex* V, double complex out[4]) {
  out[0] = conj(V[0]);
  out[1] = conj(V[2]);
  out[2] = conj(V[1]);
  out[3] = conj(V[3]);
}

/* ------------------------------------------------------------------ */
/* taper: Kaiser-Bessel via the power series of I0                      */
/* ------------------------------------------------------------------ */

/* I0(x) = sum_k ((x/2)^k / k!)^2, all terms positive so no cancellation */
double oracle_bessel_i0(double x) {
  double half = 0.5 * x, term = 1.0, sum = 1.0;
  for (int k = 1; k < 500; ++k) {
    term *= half / (double)k;
    double t2 = term * term;
    sum += t2;
    if (t2 < 1e-18 * sum) break;
  }
  return sum;
}

/* T_i for i in [0,L): kind 0 = Kaiser-Bessel with parameter beta evaluated at
 * x = 2 l_i / FOV = (2i - L)/L; kind 1 = user table copied verbatim. */
int oracle_taper(int L, int kind, double beta, const double* user, double* out) {
  if (L <= 0) return OR_ERR_INVALID;
  if (kind == 1) {
    if (!user) return OR_ERR_INVALID;
    for (int i = 0; i < L; ++i) out[i] = user[i];
    return OR_OK;
  }
  if (kind != 0) return OR_ERR_INVALID;
  double norm = oracle_bessel_i0(beta);
  for (int i = 0; i < L; ++i) {
    double x = (double)(2 * i - L) / (double)L;
    double r = 1.0 - x * x;
    out[i] = (r > 0.0 ? oracle_bessel_i0(beta * sqrt(r)) : 1.0) / norm;
  }
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* A-term interpolation                                                 */
/* ------------------------------------------------------------------ */

/* Bilinear interpolation of one station's coarse Jones samples
 * A[node_m][node_l][4] (nodes x nodes over [-FOV/2, FOV/2]) at subgrid pixel
 * (i,j).  Node a sits at l = -FOV/2 + a FOV/(nodes-1); pixel i at
 * l_i = (i-L/2) FOV/L, i.e. at fractional node (nodes-1) i / L. */
static void or_interp(const cplx* A, int nodes, int L, int i, int j, cplx out[4]) {
  double gx = (double)(nodes - 1) * (double)i / (double)L;
  double gy = (double)(nodes - 1) * (double)j / (double)L;
  int ax = (int)floor(gx), ay = (int)floor(gy);
  if (ax > nodes - 2) ax = nodes - 2;
  if (ay > nodes - 2) ay = nodes - 2;
  double fx = gx - ax, fy = gy - ay;
  const cplx* a00 = A + ((size_t)ay * nodes + ax) * 4;
  const cplx* a01 = A + ((size_t)ay * nodes + ax + 1) * 4;
  const cplx* a10 = A + ((size_t)(ay + 1) * nodes + ax) * 4;
  const cplx* a11 = A + ((size_t)(ay + 1) * nodes + ax + 1) * 4;
  for (int e = 0; e < 4; ++e)
    out[e] = (1 - fx) * (1 - fy) * a00[e] + fx * (1 - fy) * a01[e] +
             (1 - fx) * fy * a10[e] + fx * fy * a11[e];
}

/* exported for pins: interpolate a whole L x L image [j][i][4] */
int oracle_aterm_interp(int nodes, int L, const double* A_ri, double* out_ri) {
  if (nodes < 2 || L <= 0) return OR_ERR_INVALID;
  const cplx* A = (const cplx*)A_ri;
  cplx* out = (cplx*)out_ri;
  for (int j = 0; j < L; ++j)
    for (int i = 0; i < L; ++i) or_interp(A, nodes, L, i, j, out + ((size_t)j * L + i) * 4);
  return OR_OK;
}

/* 2x2 Jones helpers, row-major [00 01; 10 11] */
static void or_mul(const cplx a[4], const cplx b[4], cplx c[4]) {
  cplx r0 = a[0] * b[0] + a[1] * b[2];
  cplx r1 = a[0] * b[1] + a[1] * b[3];
  cplx r2 = a[2] * b[0] + a[3] * b[2];
  cplx r3 = a[2] * b[1] + a[3] * b[3];
  c[0] = r0; c[1] = r1; c[2] = r2; c[3] = r3;
}
static void or_herm(const cplx a[4], cplx h[4]) {
  cplx t1 = conj(a[1]), t2 = conj(a[2]);
  h[0] = conj(a[0]); h[1] = t2; h[2] = t1; h[3] = conj(a[3]);
}

/* ------------------------------------------------------------------ */
/* partitioner (Section 3.1, Section 3.3 A-term constraint)             */
/* ------------------------------------------------------------------ */

typedef struct {
  int b, blk, ts, te, c0, c1, key;
} or_sub;

static int or_cmp_sub(const void* pa, const void* pb) {
  const or_sub* a = (const or_sub*)pa;
  const or_sub* b = (const or_sub*)pb;
  if (a->b != b->b) return a->b < b->b ? -1 : 1;
  if (a->blk != b->blk) return a->blk < b->blk ? -1 : 1;
  if (a->ts != b->ts) return a->ts < b->ts ? -1 : 1;
  if (a->c0 != b->c0) return a->c0 < b->c0 ? -1 : 1;
  return 0;
}

typedef struct {
  const double* uvw;
  const double* freqs;
  int n_t, N;
  double fov;
  int layered;     /* w layers in use */
  double w_step;   /* layer width 2 w_max (wavelengths) */
} or_ctx;

/* -1 when row (b, t) is mirrored (w layers and w < 0), else +1 */
static double or_sign(const or_ctx* cx, int b, int t) {
  return cx->layered && cx->uvw[((size_t)b * cx->n_t + t) * 3 + 2] < 0.0 ? -1.0 : 1.0;
}

/* w layer key of a visibility: 2k + m, m = 1 for a mirrored row, and k the
 * layer of its gridded w' = |w| >= 0: k = floor(w' / (2 w_max)), so that
 * w0 = (2k+1) w_max and |w' - w0| <= w_max.  Members of one subgrid share
 * the key (one layer, one side).  0 when layers are off. */
static int or_layer(const or_ctx* cx, int b, int t, int c) {
  if (!cx->layered) return 0;
  double sgn = or_sign(cx, b, t);
  double w = or_wavelengths(cx->uvw, cx->n_t, b, t, 2, sgn, cx->freqs[c]);
  int k = (int)floor(w / cx->w_step);
  return 2 * k + (sgn < 0.0 ? 1 : 0);
}

/* bounding-box extent test: does the set of (t,ch) points fit within `span`
 * pixels in both the u and the v direction? */
static int or_box_fits(const or_ctx* cx, int b, const int* ts, const int* cs, int npts, double span) {
  double xlo = 0, xhi = 0, ylo = 0, yhi = 0;
  for (int n = 0; n < npts; ++n) {
    double f = cx->freqs[cs[n]];
    double sgn = or_sign(cx, b, ts[n]);
    double x = or_pix(cx->uvw, cx->n_t, b, ts[n], 0, sgn, f, cx->fov, cx->N);
    double y = or_pix(cx->uvw, cx->n_t, b, ts[n], 1, sgn, f, cx->fov, cx->N);
    if (n == 0 || x < xlo) xlo = x;
    if (n == 0 || x > xhi) xhi = x;
    if (n == 0 || y < ylo) ylo = y;
    if (n == 0 || y > yhi) yhi = y;
  }
  return (xhi - xlo) <= span && (yhi - ylo) <= span;
}

/* every visibility of the subtable [ts,te) x [c0,c1) inside the box, and in
 * layer k0? */
static int or_members_fit(const or_ctx* cx, int b, int ts, int te, int c0, int c1, double span, int k0) {
  double xlo = 0, xhi = 0, ylo = 0, yhi = 0;
  int first = 1;
  for (int t = ts; t < te; ++t)
    for (int c = c0; c < c1; ++c) {
      if (or_layer(cx, b, t, c) != k0) return 0;
      double f = cx->freqs[c];
      double sgn = or_sign(cx, b, t);
      double x = or_pix(cx->uvw, cx->n_t, b, t, 0, sgn, f, cx->fov, cx->N);
      double y = or_pix(cx->uvw, cx->n_t, b, t, 1, sgn, f, cx->fov, cx->N);
      if (first || x < xlo) xlo = x;
      if (first || x > xhi) xhi = x;
      if (first || y < ylo) ylo = y;
      if (first || y > yhi) yhi = y;
      first = 0;
    }
  return (xhi - xlo) <= span && (yhi - ylo) <= span;
}

/*
 * oracle_plan: partition every baseline's time x channel table into subtables.
 *
 * Reading of Section 3.1 (the paper gives the idea, not the constants):
 *   S  = L - P - 4           admissible pixel span of one subgrid (the -4
 *                            absorbs the flooring of the subgrid centre)
 *   G  = max(2, floor(S/4))  room left to grow in time (the fit margin)
 *   Sc = S - G               span allowed when splitting channels
 * For each baseline and each time block (the whole baseline, or each A-term
 * interval when OR_FLAG_SPLIT_INTERVALS is set) a LIFO stack of pending
 * subtables (t_start, c0, c1) starts with (block start, 0, n_ch).  A popped
 * entry is split at t_start into maximal channel ranges whose two end
 * channels span <= Sc (channels ascend, so the ends bound the range); each
 * range is grown in time while the four corners span <= S, shrunk while any
 * member falls outside S, emitted, and its remaining timesteps pushed back.
 * Output is sorted by (baseline, block, t_start, c0).
 * Placement: x0 = floor((xi_min + xi_max)/2) - L/2, likewise y0; a subgrid
 * outside [0, N-L] is an error, or is dropped with OR_FLAG_DROP.
 * Segments: one per A-term interval that intersects the subgrid's timesteps.
 * w check (reading of the Section 2.4 footnote): the w fringe across the
 * subgrid, |w - w0| * max|grad n'| * FOV pixels, must not exceed P/2 - 1,
 * i.e. |w - w0| <= w_max = (P/2 - 1) / (max|grad n'| FOV).  Without
 * OR_FLAG_W_LAYERS every subgrid has w0 = 0 and a larger |w| is an error.
 * With it (Section 2.4: the hybrid with w-stacking) rows with w < 0 are
 * mirrored (footnote of Section 2.4; see the conventions above), the gridded
 * w' >= 0 falls in layer k = floor(w' / (2 w_max)) with w0 = (2k+1) w_max,
 * one of {w_max, 3 w_max, 5 w_max, ...}, and every member of a subgrid
 * shares the layer and the side (mirrored or not) of the run's first
 * visibility: the channel runs, the time growth (corners) and the final
 * shrink (all members) also require it.  Pixel coordinates of mirrored rows
 * are those of (-u, -v).
 *
 * out_sg: cap_sg rows of 8 ints {b, t0, t1, c0, c1, x0, y0, dropped}
 * out_seg: cap_seg rows of 4 ints {subgrid, interval, t_begin, t_end}
 * out_layer (optional): per subgrid its layer k, w0 = (k + 1/2) w_step
 * out_conj (optional): per subgrid 1 if it holds mirrored rows, else 0
 * w_step_out (optional): the layer width 2 w_max in wavelengths
 */
int oracle_plan(int N, int L, int P, double fov, int flags, int n_bl, int n_t, int n_ch,
                const double* uvw, const double* freqs, const int* aterm_offsets, int n_int,
                int* out_sg, int cap_sg, int* n_sg_out, int* out_seg, int cap_seg, int* n_seg_out,
                int* out_layer, int* out_conj, double* w_step_out) {
  if (N <= 0 || L <= 0 || P < 0 || L > N || (N % 2) || (L % 2) || (P % 2) || n_bl < 0 || n_t < 0 ||
      n_ch < 0 || n_int < 1 || !(fov > 0.0))
    return OR_ERR_INVALID;
  if (aterm_offsets[0] != 0 || aterm_offsets[n_int] != n_t) return OR_ERR_INVALID;
  for (int a = 0; a < n_int; ++a)
    if (aterm_offsets[a + 1] < aterm_offsets[a]) return OR_ERR_INVALID;
  for (int c = 1; c < n_ch; ++c)
    if (!(freqs[c] > freqs[c - 1])) return OR_ERR_UNSORTED_FREQ;
  double r2max = 0.5 * fov * fov; /* corner pixel l = m = -FOV/2 */
  if (!(r2max < 1.0)) return OR_ERR_INVALID;
  int S = L - P - 4;
  if (S < 1) return OR_ERR_INVALID;
  int G = S / 4 > 2 ? S / 4 : 2;
  int Sc = S - G;
  if (Sc < 0) Sc = 0;

  /* w limit */
  double gmax = sqrt(r2max) / sqrt(1.0 - r2max);
  double wlim = 0.5 * P - 1.0;
  const int layered = (flags & OR_FLAG_W_LAYERS) != 0;
  const double w_step = 2.0 * (wlim / (gmax * fov));
  if (w_step_out) *w_step_out = w_step;
  if (layered && !(w_step > 0.0)) return OR_ERR_INVALID;
  for (int b = 0; b < n_bl && !layered; ++b)
    for (int t = 0; t < n_t; ++t)
      for (int c = 0; c < n_ch; ++c) {
        double w = or_wavelengths(uvw, n_t, b, t, 2, 1.0, freqs[c]);
        if (fabs(w) * gmax * fov > wlim) return OR_ERR_W_TOO_LARGE;
      }

  or_ctx cx = {uvw, freqs, n_t, N, fov, layered, w_step};
  int n_sg = 0, n_seg = 0;
  int stack_cap = 64;
  int* stack = (int*)malloc(sizeof(int) * 3 * stack_cap);
  int list_cap = 64;
  or_sub* list = (or_sub*)malloc(sizeof(or_sub) * list_cap);
  int status = OR_OK;

  for (int b = 0; b < n_bl && status == OR_OK; ++b) {
    int nblk = (flags & OR_FLAG_SPLIT_INTERVALS) ? n_int : 1;
    int n_list = 0;
    for (int blk = 0; blk < nblk; ++blk) {
      int ta = (flags & OR_FLAG_SPLIT_INTERVALS) ? aterm_offsets[blk] : 0;
      int tb = (flags & OR_FLAG_SPLIT_INTERVALS) ? aterm_offsets[blk + 1] : n_t;
      if (ta >= tb || n_ch == 0) continue;
      int sp = 0;
      stack[0] = ta; stack[1] = 0; stack[2] = n_ch; sp = 1;
      while (sp > 0) {
        --sp;
        int ts = stack[3 * sp], c0 = stack[3 * sp + 1], c1 = stack[3 * sp + 2];
        int c = c0;
        while (c < c1) {
          int k0 = or_layer(&cx, b, ts, c);
          int hi = c + 1; /* range is [c, hi) */
          for (;;) {
            if (hi >= c1) break;
            int tt[2] = {ts, ts}, cc[2] = {c, hi};
            if (!or_box_fits(&cx, b, tt, cc, 2, (double)Sc)) break;
            if (or_layer(&cx, b, ts, hi) != k0) break;
            ++hi;
          }
          int te = ts + 1;
          for (;;) {
            if (te >= tb) break;
            int tt[4] = {ts, ts, te, te}, cc[4] = {c, hi - 1, c, hi - 1};
            if (!or_box_fits(&cx, b, tt, cc, 4, (double)S)) break;
            if (or_layer(&cx, b, te, c) != k0 || or_layer(&cx, b, te, hi - 1) != k0) break;
            ++te;
          }
          while (te > ts + 1 && !or_members_fit(&cx, b, ts, te, c, hi, (double)S, k0)) --te;
          if (n_list == list_cap) {
            list_cap *= 2;
            list = (or_sub*)realloc(list, sizeof(or_sub) * list_cap);
          }
          or_sub s = {b, blk, ts, te, c, hi, k0};
          list[n_list++] = s;
          if (te < tb) {
            if (sp == stack_cap) {
              stack_cap *= 2;
              stack = (int*)realloc(stack, sizeof(int) * 3 * stack_cap);
            }
            stack[3 * sp] = te; stack[3 * sp + 1] = c; stack[3 * sp + 2] = hi; ++sp;
          }
          c = hi;
        }
      }
    }
    qsort(list, n_list, sizeof(or_sub), or_cmp_sub);
    for (int n = 0; n < n_list; ++n) {
      or_sub s = list[n];
      /* exact bounding box of the members (mirrored coordinates for mirrored rows) */
      double xlo = 0, xhi = 0, ylo = 0, yhi = 0;
      int first = 1;
      for (int t = s.ts; t < s.te; ++t)
        for (int c = s.c0; c < s.c1; ++c) {
          double f = freqs[c];
          double sgn = or_sign(&cx, b, t);
          double x = or_pix(uvw, n_t, b, t, 0, sgn, f, fov, N);
          double y = or_pix(uvw, n_t, b, t, 1, sgn, f, fov, N);
          if (first || x < xlo) xlo = x;
          if (first || x > xhi) xhi = x;
          if (first || y < ylo) ylo = y;
          if (first || y > yhi) yhi = y;
          first = 0;
        }
      int x0 = (int)floor((xlo + xhi) / 2.0) - L / 2;
      int y0 = (int)floor((ylo + yhi) / 2.0) - L / 2;
      int dropped = 0;
      if (x0 < 0 || y0 < 0 || x0 + L > N || y0 + L > N) {
        if (!(flags & OR_FLAG_DROP)) { status = OR_ERR_OUT_OF_GRID; break; }
        dropped = 1;
      }
      if (n_sg >= cap_sg) { status = OR_ERR_CAPACITY; break; }
      int* row = out_sg + (size_t)n_sg * 8;
      row[0] = b; row[1] = s.ts; row[2] = s.te; row[3] = s.c0; row[4] = s.c1;
      row[5] = x0; row[6] = y0; row[7] = dropped;
      if (out_layer) out_layer[n_sg] = s.key >> 1;
      if (out_conj) out_conj[n_sg] = s.key & 1;
      for (int a = 0; a < n_int; ++a) {
        int lo = aterm_offsets[a] > s.ts ? aterm_offsets[a] : s.ts;
        int hi = aterm_offsets[a + 1] < s.te ? aterm_offsets[a + 1] : s.te;
        if (lo >= hi) continue;
        if (n_seg >= cap_seg) { status = OR_ERR_CAPACITY; break; }
        int* sr = out_seg + (size_t)n_seg * 4;
        sr[0] = n_sg; sr[1] = a; sr[2] = lo; sr[3] = hi;
        ++n_seg;
      }
      if (status != OR_OK) break;
      ++n_sg;
    }
  }
  free(stack);
  free(list);
  *n_sg_out = n_sg;
  *n_seg_out = n_seg;
  return status;
}

/* ------------------------------------------------------------------ */
/* the centred L-point DFT used for the subgrid transform (Eq. 8)       */
/* ------------------------------------------------------------------ */

/* matrix F[x][i] = exp(sign * 2 pi i (x-L/2)(i-L/2) / L).  The integer
 * product is reduced modulo L first: the exponential is L-periodic in it. */
static cplx* or_dft_matrix(int L, int sign) {
  cplx* F = (cplx*)malloc(sizeof(cplx) * (size_t)L * L);
  for (int x = 0; x < L; ++x)
    for (int i = 0; i < L; ++i) {
      long long prod = (long long)(x - L / 2) * (long long)(i - L / 2);
      long long r = prod % L;
      if (r < 0) r += L;
      double ang = sign * 2.0 * OR_PI * (double)r / (double)L;
      F[(size_t)x * L + i] = cos(ang) + I * sin(ang);
    }
  return F;
}

/* out[y][x] = sum_{j,i} F[y][j] F[x][i] in[j][i]  for one L x L plane */
static void or_dft2_plane(int L, const cplx* F, const cplx* in, cplx* out, cplx* tmp) {
  for (int j = 0; j < L; ++j)
    for (int x = 0; x < L; ++x) {
      cplx s = 0;
      for (int i = 0; i < L; ++i) s += F[(size_t)x * L + i] * in[(size_t)j * L + i];
      tmp[(size_t)j * L + x] = s;
    }
  for (int y = 0; y < L; ++y)
    for (int x = 0; x < L; ++x) {
      cplx s = 0;
      for (int j = 0; j < L; ++j) s += F[(size_t)y * L + j] * tmp[(size_t)j * L + x];
      out[(size_t)y * L + x] = s;
    }
}

/* exported for pins: centred 2-D DFT of n_planes L x L planes, sign = -1
 * (forward, gridding) or +1 (inverse, degridding), unnormalised. */
int oracle_dft2(int L, int sign, int n_planes, const double* in_ri, double* out_ri) {
  if (L <= 0 || (L % 2) || (sign != 1 && sign != -1)) return OR_ERR_INVALID;
  cplx* F = or_dft_matrix(L, sign);
  cplx* tmp = (cplx*)malloc(sizeof(cplx) * (size_t)L * L);
  for (int p = 0; p < n_planes; ++p)
    or_dft2_plane(L, F, (const cplx*)in_ri + (size_t)p * L * L, (cplx*)out_ri + (size_t)p * L * L, tmp);
  free(tmp);
  free(F);
  return OR_OK;
}

/* ------------------------------------------------------------------ */
/* gridding and degridding                                              */
/* ------------------------------------------------------------------ */

typedef struct {
  int N, L, P;
  double fov;
  int taper_kind;
  double beta;
  const double* taper_user;
  int nodes;
  int n_st, n_bl, n_t, n_ch;
  const int* baselines;
  const double* uvw;
  const double* freqs;
  int n_int;
  const int* sg;
  int n_sg;
  const int* seg;
  int n_seg;
  const int* layer;  /* per subgrid w layer k (NULL: no layers, w0 = 0) */
  const int* conj;   /* per subgrid 1 = mirrored rows (NULL: none) */
  double w_step;     /* w0 = (k + 1/2) w_step */
  int k_min;         /* the master grid holds layers k_min .. k_min + n_layers - 1 */
} or_job;

/* n'(l,m) = sqrt(1 - l^2 - m^2) - 1 */
static double or_nprime(double l, double m) { return sqrt(1.0 - l * l - m * m) - 1.0; }

/* subgrid image X (Eq. 10 with the deferred A-term of Section 3.3), all 4
 * polarisations, layout [pol][j][i].
 * With normalize (the A-term power normalisation of Section 3.3): each
 * segment's corrected image A_p^H X A_q is divided, pixel by pixel, by the
 * Frobenius norm f = ||A_p^H A_q||_F of the product of the two matrices the
 * gridder applies (A_1^{-1} (A_2^{-1})^H in the paper's notation, where the
 * caller passes inverse terms), and wsub[j L + i] accumulates n_seg / f,
 * n_seg the segment's visibility count.  A pixel with f = 0 contributes
 * nothing and no weight. */
static void or_subgrid_image(const or_job* jb, int s, const cplx* vis, const cplx* aterms,
                             const double* T, const int* seg_first, const int* seg_count, cplx* X,
                             int normalize, double* wsub) {
  const int L = jb->L, N = jb->N, nodes = jb->nodes;
  const int* row = jb->sg + (size_t)s * 8;
  int b = row[0], c0 = row[3], c1 = row[4], x0 = row[5], y0 = row[6];
  /* a mirrored subgrid grids V^H of baseline (q, p) at (-u, -v, -w) */
  int mirrored = jb->conj ? jb->conj[s] : 0;
  double sgn = mirrored ? -1.0 : 1.0;
  int p = jb->baselines[2 * b + (mirrored ? 1 : 0)], q = jb->baselines[2 * b + (mirrored ? 0 : 1)];
  double u0 = (double)(x0 + L / 2 - N / 2) / jb->fov;
  double v0 = (double)(y0 + L / 2 - N / 2) / jb->fov;
  double w0 = jb->layer ? ((double)jb->layer[s] + 0.5) * jb->w_step : 0.0;
  memset(X, 0, sizeof(cplx) * 4 * (size_t)L * L);
  for (int g = seg_first[s]; g < seg_first[s] + seg_count[s]; ++g) {
    const int* sr = jb->seg + (size_t)g * 4;
    int a = sr[1], tb = sr[2], te = sr[3];
    const cplx* Ap = aterms + ((size_t)a * jb->n_st + p) * nodes * nodes * 4;
    const cplx* Aq = aterms + ((size_t)a * jb->n_st + q) * nodes * nodes * 4;
    for (int j = 0; j < L; ++j)
      for (int i = 0; i < L; ++i) {
        double l = (double)(i - L / 2) * jb->fov / (double)L;
        double m = (double)(j - L / 2) * jb->fov / (double)L;
        double n1 = or_nprime(l, m);
        cplx acc[4] = {0, 0, 0, 0};
        for (int t = tb; t < te; ++t)
          for (int c = c0; c < c1; ++c) {
            double f = jb->freqs[c];
            double u = or_wavelengths(jb->uvw, jb->n_t, b, t, 0, sgn, f);
            double v = or_wavelengths(jb->uvw, jb->n_t, b, t, 1, sgn, f);
            double w = or_wavelengths(jb->uvw, jb->n_t, b, t, 2, sgn, f);
            double phi = (u - u0) * l + (v - v0) * m + (w - w0) * n1;
            cplx e = cexp(I * 2.0 * OR_PI * phi);
            const cplx* V = vis + (((size_t)b * jb->n_t + t) * jb->n_ch + c) * 4;
            cplx Vm[4];
            if (mirrored) or_vis_herm(V, Vm);
            else memcpy(Vm, V, sizeof Vm);
            for (int e4 = 0; e4 < 4; ++e4) acc[e4] += Vm[e4] * e;
          }
        cplx Api[4], Aqi[4], ApH[4], M[4], E[4];
        or_interp(Ap, nodes, L, i, j, Api);
        or_interp(Aq, nodes, L, i, j, Aqi);
        or_herm(Api, ApH);
        or_mul(acc, Aqi, M);
        or_mul(ApH, M, E);
        double tt = T[i] * T[j];
        if (normalize) {
          cplx Pm[4];
          or_mul(ApH, Aqi, Pm);
          double f2 = 0.0;
          for (int e4 = 0; e4 < 4; ++e4) f2 += creal(Pm[e4]) * creal(Pm[e4]) + cimag(Pm[e4]) * cimag(Pm[e4]);
          double f = sqrt(f2);
          if (f > 0.0) {
            tt /= f;
            wsub[(size_t)j * L + i] += (double)((te - tb) * (c1 - c0)) / f;
          } else {
            tt = 0.0;
          }
        }
        for (int e4 = 0; e4 < 4; ++e4) X[((size_t)e4 * L + j) * L + i] += tt * E[e4];
      }
  }
}

static void or_seg_index(const or_job* jb, int* seg_first, int* seg_count) {
  for (int s = 0; s < jb->n_sg; ++s) { seg_first[s] = 0; seg_count[s] = 0; }
  for (int g = jb->n_seg - 1; g >= 0; --g) {
    int s = jb->seg[(size_t)g * 4];
    seg_first[s] = g;
    seg_count[s] += 1;
  }
}

/*
 * oracle_grid: grid all non-dropped subgrids into grid[4][N][N] (accumulated).
 * vis: complex [n_bl][n_t][n_ch][4]; aterms: complex [n_int][n_st][nodes][nodes][4].
 * subgrid_images (optional): complex [n_sg][4][L][L], the subgrid images X
 * before the FFT; subgrid_uv (optional): the same after the FFT.
 * With w layers (layer != NULL) subgrid s uses w0 = (layer[s] + 1/2) w_step
 * in its phase and is added into grid[layer[s] - k_min][4][N][N]; conj
 * (optional) marks the mirrored subgrids.
 * npol: 4 (correlation planes) or 1 (Stokes I): with 1 the grid holds
 * one plane per layer, I = (XX + YY) / 2 of each corrected subgrid image,
 * and the subgrid image outputs hold that one plane.
 * normalize: A-term power normalisation (see or_subgrid_image); weights
 * (needed with normalize) double [L*L + 1] accumulates, over the non-dropped
 * subgrids, sum n_seg / f per subgrid pixel and in its last slot sum n_seg.
 */
int oracle_grid(int N, int L, int P, double fov, int taper_kind, double beta, const double* taper_user,
                int nodes, int n_st, int n_bl, int n_t, int n_ch, const int* baselines, const double* uvw,
                const double* freqs, int n_int, const int* sg, int n_sg, const int* seg, int n_seg,
                const int* layer, const int* conj, double w_step, int k_min, int npol,
                const double* vis_ri, const double* aterms_ri, double* grid_ri, double* subgrid_images,
                double* subgrid_uv, int normalize, double* weights) {
  or_job jb = {N, L, P, fov, taper_kind, beta, taper_user, nodes, n_st, n_bl, n_t, n_ch, baselines,
               uvw, freqs, n_int, sg, n_sg, seg, n_seg, layer, conj, w_step, k_min};
  double* T = (double*)malloc(sizeof(double) * L);
  int st = oracle_taper(L, taper_kind, beta, taper_user, T);
  if (st) { free(T); return st; }
  int* seg_first = (int*)malloc(sizeof(int) * (n_sg > 0 ? n_sg : 1));
  int* seg_count = (int*)malloc(sizeof(int) * (n_sg > 0 ? n_sg : 1));
  or_seg_index(&jb, seg_first, seg_count);
  cplx* F = or_dft_matrix(L, -1);
  const cplx* vis = (const cplx*)vis_ri;
  const cplx* aterms = (const cplx*)aterms_ri;
  cplx* grid = (cplx*)grid_ri;
  const size_t plane = (size_t)L * L;
  if ((npol != 1 && npol != 4) || (normalize && !weights)) {
    free(T);
    free(seg_first);
    free(seg_count);
    free(F);
    return OR_ERR_INVALID;
  }
  const int batch = 64;
  cplx* buf = (cplx*)malloc(sizeof(cplx) * 4 * plane * batch);
  double* wbuf = (double*)calloc(plane * batch, sizeof(double));
  for (int s0 = 0; s0 < n_sg; s0 += batch) {
    int nb = n_sg - s0 < batch ? n_sg - s0 : batch;
    memset(wbuf, 0, sizeof(double) * plane * batch);
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = 0; k < nb; ++k) {
      int s = s0 + k;
      cplx* X = (cplx*)malloc(sizeof(cplx) * 4 * plane);
      cplx* tmp = (cplx*)malloc(sizeof(cplx) * plane);
      or_subgrid_image(&jb, s, vis, aterms, T, seg_first, seg_count, X, normalize, wbuf + (size_t)k * plane);
      if (npol == 1) /* Stokes I = (XX + YY) / 2 of the corrected image */
        for (size_t e = 0; e < plane; ++e) X[e] = 0.5 * (X[e] + X[3 * plane + e]);
      if (subgrid_images) memcpy((cplx*)subgrid_images + (size_t)s * npol * plane, X, sizeof(cplx) * npol * plane);
      for (int e = 0; e < npol; ++e) or_dft2_plane(L, F, X + e * plane, buf + ((size_t)k * 4 + e) * plane, tmp);
      if (subgrid_uv) memcpy((cplx*)subgrid_uv + (size_t)s * npol * plane, buf + (size_t)k * 4 * plane, sizeof(cplx) * npol * plane);
      free(tmp);
      free(X);
    }
    /* adder, in subgrid order */
    for (int k = 0; k < nb; ++k) {
      const int* row = sg + (size_t)(s0 + k) * 8;
      if (row[7]) continue;
      int x0 = row[5], y0 = row[6];
      cplx* gl = grid + (layer ? (size_t)(layer[s0 + k] - k_min) * npol * N * N : 0);
      for (int e = 0; e < npol; ++e)
        for (int y = 0; y < L; ++y)
          for (int x = 0; x < L; ++x)
            gl[((size_t)e * N + (y0 + y)) * N + (x0 + x)] += buf[(((size_t)k * 4 + e) * L + y) * L + x];
      if (normalize) {
        for (size_t e = 0; e < plane; ++e) weights[e] += wbuf[(size_t)k * plane + e];
        int c0 = row[3], c1 = row[4];
        for (int g = seg_first[s0 + k]; g < seg_first[s0 + k] + seg_count[s0 + k]; ++g)
          weights[plane] += (double)((seg[(size_t)g * 4 + 3] - seg[(size_t)g * 4 + 2]) * (c1 - c0));
      }
    }
  }
  free(wbuf);
  free(buf);
  free(F);
  free(seg_first);
  free(seg_count);
  free(T);
  return OR_OK;
}

/*
 * oracle_degrid: predict visibilities from grid[4][N][N] (Eq. 13 read as the
 * adjoint of the gridder).  vis_out is overwritten; visibilities of dropped
 * subgrids are zero.  With w layers, subgrid s reads grid[layer[s] - k_min]
 * and uses w0 = (layer[s] + 1/2) w_step; a mirrored subgrid predicts the
 * mirror (baseline (q, p) at (-u, -v, -w)) and stores its conjugate
 * transpose.  npol = 1: the grid holds Stokes I and the
 * model is unpolarised, Y = Y_I times the 2x2 identity (XX = YY = I).
 */
int oracle_degrid(int N, int L, int P, double fov, int taper_kind, double beta, const double* taper_user,
                  int nodes, int n_st, int n_bl, int n_t, int n_ch, const int* baselines, const double* uvw,
                  const double* freqs, int n_int, const int* sg, int n_sg, const int* seg, int n_seg,
                  const int* layer, const int* conj, double w_step, int k_min, int npol,
                  const double* grid_ri, const double* aterms_ri, double* vis_ri) {
  or_job jb = {N, L, P, fov, taper_kind, beta, taper_user, nodes, n_st, n_bl, n_t, n_ch, baselines,
               uvw, freqs, n_int, sg, n_sg, seg, n_seg, layer, conj, w_step, k_min};
  if (npol != 1 && npol != 4) return OR_ERR_INVALID;
  double* T = (double*)malloc(sizeof(double) * L);
  int st = oracle_taper(L, taper_kind, beta, taper_user, T);
  if (st) { free(T); return st; }
  int* seg_first = (int*)malloc(sizeof(int) * (n_sg > 0 ? n_sg : 1));
  int* seg_count = (int*)malloc(sizeof(int) * (n_sg > 0 ? n_sg : 1));
  or_seg_index(&jb, seg_first, seg_count);
  cplx* F = or_dft_matrix(L, +1);
  const cplx* grid = (const cplx*)grid_ri;
  const cplx* aterms = (const cplx*)aterms_ri;
  cplx* vis = (cplx*)vis_ri;
  memset(vis, 0, sizeof(cplx) * 4 * (size_t)n_bl * n_t * n_ch);
  const size_t plane = (size_t)L * L;
#pragma omp parallel for schedule(dynamic, 1)
  for (int s = 0; s < n_sg; ++s) {
    const int* row = sg + (size_t)s * 8;
    if (row[7]) continue;
    int b = row[0], c0 = row[3], c1 = row[4], x0 = row[5], y0 = row[6];
    int mirrored = conj ? conj[s] : 0;
    double sgn = mirrored ? -1.0 : 1.0;
    int p = baselines[2 * b + (mirrored ? 1 : 0)], q = baselines[2 * b + (mirrored ? 0 : 1)];
    cplx* Yh = (cplx*)malloc(sizeof(cplx) * 4 * plane);
    cplx* Y = (cplx*)malloc(sizeof(cplx) * 4 * plane);
    cplx* tmp = (cplx*)malloc(sizeof(cplx) * plane);
    /* splitter */
    const cplx* gl = grid + (layer ? (size_t)(layer[s] - k_min) * npol * N * N : 0);
    for (int e = 0; e < npol; ++e)
      for (int y = 0; y < L; ++y)
        for (int x = 0; x < L; ++x)
          Yh[((size_t)e * L + y) * L + x] = gl[((size_t)e * N + (y0 + y)) * N + (x0 + x)];
    for (int e = 0; e < npol; ++e) or_dft2_plane(L, F, Yh + e * plane, Y + e * plane, tmp);
    if (npol == 1) /* Stokes-I model: Y = Y_I times the 2x2 identity */
      for (size_t e = 0; e < plane; ++e) {
        Y[plane + e] = 0.0;
        Y[2 * plane + e] = 0.0;
        Y[3 * plane + e] = Y[e];
      }
    double u0 = (double)(x0 + L / 2 - N / 2) / fov;
    double v0 = (double)(y0 + L / 2 - N / 2) / fov;
    double w0 = layer ? ((double)layer[s] + 0.5) * w_step : 0.0;
    for (int g = seg_first[s]; g < seg_first[s] + seg_count[s]; ++g) {
      const int* sr = seg + (size_t)g * 4;
      int a = sr[1], tb = sr[2], te = sr[3];
      const cplx* Ap = aterms + ((size_t)a * n_st + p) * nodes * nodes * 4;
      const cplx* Aq = aterms + ((size_t)a * n_st + q) * nodes * nodes * 4;
      /* Z = T_i T_j A_p Y A_q^H on every pixel */
      cplx* Z = (cplx*)malloc(sizeof(cplx) * 4 * plane);
      for (int j = 0; j < L; ++j)
        for (int i = 0; i < L; ++i) {
          cplx Api[4], Aqi[4], AqH[4], Yp[4], M[4], E[4];
          or_interp(Ap, nodes, L, i, j, Api);
          or_interp(Aq, nodes, L, i, j, Aqi);
          or_herm(Aqi, AqH);
          for (int e4 = 0; e4 < 4; ++e4) Yp[e4] = Y[((size_t)e4 * L + j) * L + i];
          or_mul(Api, Yp, M);
          or_mul(M, AqH, E);
          double tt = T[i] * T[j];
          for (int e4 = 0; e4 < 4; ++e4) Z[((size_t)j * L + i) * 4 + e4] = tt * E[e4];
        }
      for (int t = tb; t < te; ++t)
        for (int c = c0; c < c1; ++c) {
          double f = freqs[c];
          double u = or_wavelengths(uvw, n_t, b, t, 0, sgn, f);
          double v = or_wavelengths(uvw, n_t, b, t, 1, sgn, f);
          double w = or_wavelengths(uvw, n_t, b, t, 2, sgn, f);
          cplx acc[4] = {0, 0, 0, 0};
          for (int j = 0; j < L; ++j)
            for (int i = 0; i < L; ++i) {
              double l = (double)(i - L / 2) * fov / (double)L;
              double m = (double)(j - L / 2) * fov / (double)L;
              double phi = (u - u0) * l + (v - v0) * m + (w - w0) * or_nprime(l, m);
              cplx e = cexp(-I * 2.0 * OR_PI * phi);
              const cplx* Zp = Z + ((size_t)j * L + i) * 4;
              for (int e4 = 0; e4 < 4; ++e4) acc[e4] += Zp[e4] * e;
            }
          cplx* V = vis + (((size_t)b * n_t + t) * n_ch + c) * 4;
          if (mirrored) or_vis_herm(acc, V);
          else for (int e4 = 0; e4 < 4; ++e4) V[e4] = acc[e4];
        }
      free(Z);
    }
    free(tmp);
    free(Y);
    free(Yh);
  }
  free(F);
  free(seg_first);
  free(seg_count);
  free(T);
  return OR_OK;
}
