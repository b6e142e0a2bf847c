// GES oracle -- TEST INFRASTRUCTURE ONLY.
//
// A plain, slow, FP64 CPU restatement of the Generalized Exponential Splatting
// rasterizer (Hamdi et al., "GES: Generalized Exponential Splatting for
// Efficient Radiance Field Rendering").  Only the tests, the package's smoke
// check and the benchmark's CPU-baseline leg may load it; the product path never
// does.  It shares no code, header or constant table with the CUDA library.
//
// What it computes, and which passage each part follows:
//   * GES kernel  L(x) = exp(-1/2 ((x-mu)^T Sigma^-1 (x-mu))^(beta/2))      Sec. 4.1, Eq. (ges)
//   * Sigma = R S S^T R^T with S scaled by the shape modification phi(beta)  Sec. 4.1
//   * phi_bar_rho(beta) = 2 / (1 + exp(-(rho*beta - 2*rho))), rho = 0.1     Sec. 4.2, Eq. (approx); App. B.2
//     or, as an option, the exact phi_n(beta) = 2 Gamma(3/beta)/Gamma(1/beta) Sec. 4.2, Eq. (probablity)
//   * EWA projection Sigma' = J W Sigma W^T J^T (Zwicker et al.)             Sec. 4.1
//   * discrete front-to-back compositing of the volume-rendering integral   Sec. 4.2, Eq. (transmittance)
//   * view-dependent colour from real spherical harmonics                   Sec. 4.1
// Readings where the paper is silent (alpha clamp 0.99, skip below 1/255,
// stop at T < 1e-4, 0.3 px dilation, 16x16 tiles, the beta-dependent extent,
// SH conventions, FP32 key path) are listed in the design notes and restated
// next to the code that uses them.
//
// Parts:
//   1. Key module (FP32, fixed operation order, no contraction): visibility,
//      depth key, tile rectangle.  These decide integers (which tiles a
//      primitive lands in, the sort order), so they are taken in the kernel's
//      precision, with every operation spelled out.  Compiled with
//      -ffp-contract=off.
//   2. FP64 projection, templated on the scalar type so that the same code
//      runs on doubles (rendering) and on forward-mode dual numbers (exact
//      Jacobians for the analytic backward).
//   3. Brute-force FP64 renderer: every visible primitive at every pixel,
//      global depth order, no tiles.
//   4. Tiled FP64 renderer (same per-pixel arithmetic, tile lists from part 1)
//      used only to check that tiling loses nothing.
//   5. Analytic FP64 backward: per pixel by hand (reverse order), per
//      primitive by the dual-number Jacobian of part 2.
//
// Parity pins live in tests/test_oracle_pins.py (closed forms, invariants,
// finite differences).  The exact-Gamma modification (Eq. probablity) is an option
// of the projection, normalised to 2 Gamma(3/beta) / Gamma(1/beta) so that it is 1
// at beta = 2 like phi_bar; it is applied to the scale vector (phi_mode 1) or, read
// as a variance ratio, to the variance (phi_mode 2).

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <thread>
#include <vector>

namespace {

// ---------------------------------------------------------------------------
// camera / parameter blocks (flat double arrays from Python)
// ---------------------------------------------------------------------------
struct Cam {
  int W, H;
  double fx, fy, cx, cy;
  double V[16];
  double campos[3];
  double znear;
  double bg[3];
};
struct Par {
  double rho;
  int mode;  // 0 = GEF falloff exp(-1/2 q^(beta/2)); 1 = paper's Gaussian-form rasterizer exp(-1/2 q)
  int phi_mode;  // scale modification: 0 = phi_bar_rho (Eq. approx); 1 = normalised exact phi_n on the
                 // scale vector; 2 = phi_n on the variance (sqrt(phi_n) on the scale vector)
  double dilation, alpha_max, alpha_min, t_min, margin_rel, margin_abs, clamp_fov;
  double flag_tol_alpha, flag_tol_t;
};

Cam read_cam(const double* c) {
  Cam k;
  k.W = (int)c[0];
  k.H = (int)c[1];
  k.fx = c[2]; k.fy = c[3]; k.cx = c[4]; k.cy = c[5];
  for (int i = 0; i < 16; ++i) k.V[i] = c[6 + i];
  for (int i = 0; i < 3; ++i) k.campos[i] = c[22 + i];
  k.znear = c[25];
  for (int i = 0; i < 3; ++i) k.bg[i] = c[26 + i];
  return k;
}
Par read_par(const double* p) {
  Par r;
  r.rho = p[0]; r.mode = (int)p[1]; r.dilation = p[2]; r.alpha_max = p[3]; r.alpha_min = p[4];
  r.t_min = p[5]; r.margin_rel = p[6]; r.margin_abs = p[7]; r.clamp_fov = p[8];
  r.flag_tol_alpha = p[9]; r.flag_tol_t = p[10];
  r.phi_mode = (int)p[11];
  return r;
}

constexpr int TILE = 16;

// ---------------------------------------------------------------------------
// 1. Key module, FP32.
// exp2 / log2 are spelled out (range reduction + series) so that the value is a
//    fixed function of the inputs: x = n + f, 2^f by its Taylor series in f*ln2
//    to degree 7; log2 m via atanh series of s = (m-1)/(m+1), m in [sqrt(.5), sqrt(2)).
// ---------------------------------------------------------------------------
struct FExpCoef {
  float c[8];
  FExpCoef() {
    double ln2 = std::log(2.0);
    double t = 1.0;
    for (int k = 0; k < 8; ++k) {
      if (k > 0) t = t * ln2 / (double)k;  // ln2^k / k!
      c[k] = (float)t;
    }
  }
};
const FExpCoef kExp;

float key_exp2(float x) {
  // clamp; a NaN argument maps to the upper bound
  if (!(x <= 126.0f)) x = 126.0f;
  if (!(x >= -100.0f)) x = -100.0f;
  float n = std::rint(x);
  float f = x - n;
  float p = kExp.c[7];
  for (int k = 6; k >= 0; --k) {
    p = p * f;
    p = p + kExp.c[k];
  }
  return std::ldexp(p, (int)n);
}

float key_log2(float x) {
  // x > 0, finite, normal
  uint32_t b;
  std::memcpy(&b, &x, 4);
  int e = (int)((b >> 23) & 0xffu) - 127;
  uint32_t mb = (b & 0x7fffffu) | 0x3f800000u;
  float m;
  std::memcpy(&m, &mb, 4);
  const float sqrt2 = (float)std::sqrt(2.0);
  if (m > sqrt2) {
    m = m * 0.5f;
    e = e + 1;
  }
  float s = (m - 1.0f) / (m + 1.0f);
  float s2 = s * s;
  // 1 + s2/3 + s2^2/5 + ... + s2^5/11
  float p = (float)(1.0 / 11.0);
  p = p * s2; p = p + (float)(1.0 / 9.0);
  p = p * s2; p = p + (float)(1.0 / 7.0);
  p = p * s2; p = p + (float)(1.0 / 5.0);
  p = p * s2; p = p + (float)(1.0 / 3.0);
  p = p * s2; p = p + 1.0f;
  float ln_m = (2.0f * s) * p;
  const float log2e = (float)(1.0 / std::log(2.0));
  return (float)e + ln_m * log2e;
}

// ln Gamma(x) for x > 0, FP32.  Gamma(x) = Gamma(z) / (x (x+1) ... (z-1)) with z = x + k the first
// shift at or above 4 (k <= 4), then Stirling's series for ln Gamma(z):
//   (z - 1/2) ln z - z + ln(2 pi)/2 + 1/(12 z) - 1/(360 z^3) + 1/(1260 z^5) - 1/(1680 z^7)
// (its first omitted term, 1/(1188 z^9), is below 4e-9 at z >= 4).  ln via key_log2 * ln 2.
float key_lgamma(float x) {
  const float ln2 = (float)std::log(2.0);
  float z = x, acc = 1.0f;
  for (int k = 0; k < 4 && z < 4.0f; ++k) {
    acc = acc * z;
    z = z + 1.0f;
  }
  float r = 1.0f / z;
  float r2 = r * r;
  float ser = -(float)(1.0 / 1680.0);
  ser = ser * r2; ser = ser + (float)(1.0 / 1260.0);
  ser = ser * r2; ser = ser - (float)(1.0 / 360.0);
  ser = ser * r2; ser = ser + (float)(1.0 / 12.0);
  ser = ser * r;
  float lz = key_log2(z) * ln2;
  float lg = (z - 0.5f) * lz;
  lg = lg - z;
  lg = lg + (float)(0.5 * std::log(2.0 * std::acos(-1.0)));
  lg = lg + ser;
  return lg - key_log2(acc) * ln2;
}

// The scale modification in the key path's precision:
//   mode 0: phi_bar_rho(beta) = 2 / (1 + 2^(-rho (beta - 2) log2 e))                 (Eq. approx)
//   mode 1: phi_n(beta) = 2 Gamma(3/beta) / Gamma(1/beta)
//                       = 2^((ln Gamma(3/beta) - ln Gamma(1/beta) + ln 2) log2 e)  (Eq. probablity,
//           normalised to 1 at beta = 2)
//   mode 2: sqrt(phi_n(beta)): the same exponent halved
float key_phi(float beta, float rho, int phi_mode) {
  const float log2e = (float)(1.0 / std::log(2.0));
  if (phi_mode == 0) {
    float dbeta = beta - 2.0f;
    float rdb = rho * dbeta;
    float ex = key_exp2((-rdb) * log2e);
    return 2.0f / (1.0f + ex);
  }
  float g3 = key_lgamma(3.0f / beta);
  float g1 = key_lgamma(1.0f / beta);
  float e = ((g3 - g1) + (float)std::log(2.0)) * log2e;
  if (phi_mode == 2) e = e * 0.5f;
  return key_exp2(e);
}

struct KeyOut {
  uint32_t depth_key;
  int32_t rect[4];  // x0, y0, x1, y1 (tiles, end exclusive): bounding box of the extent
  uint32_t touched; // tiles the extent actually meets (sum of the row spans)
  float mean2d[2], cov2d[3], qstar, qlim, margin_abs;
};

// Tiles of row ty met by the ellipse {d : d^T cov^-1 d <= qlim} around the 2D mean (FP32, fixed
// order, no contraction).  The row band is y in [16 ty, 16 ty + 16); within it the ellipse's
// x-extent runs from its leftmost to its rightmost point, x(dy) = (b/c) dy +- sqrt((qlim - dy^2/c)
// det/c), whose extremes over the whole ellipse lie at dy = +-b sqrt(qlim/a); over the band they lie
// at that dy clamped into the band.  The span, widened by margin_abs, is clipped to the bounding
// box's columns [rect0, rect2).  Per-primitive constants first, then one evaluation per row.
struct RowConsts {
  float Y, sl, g, ic, dys;
};
RowConsts row_consts(const KeyOut& k) {
  const float a = k.cov2d[0], b = k.cov2d[1], c = k.cov2d[2], ql = k.qlim;
  RowConsts r;
  r.Y = std::sqrt(ql * c);
  const float det = a * c - b * b;
  r.sl = b / c;
  r.g = det / c;
  r.ic = 1.0f / c;
  r.dys = b * std::sqrt(ql / a);
  return r;
}
bool row_span(const KeyOut& k, const RowConsts& rc, int ty, int& tx0, int& tx1) {
  const float u = k.mean2d[0], v = k.mean2d[1], ql = k.qlim;
  const float lo = (float)(16 * ty) - v;
  const float hi = (float)(16 * ty + 16) - v;
  const float lo2 = std::fmax(lo, -rc.Y), hi2 = std::fmin(hi, rc.Y);
  if (!(lo2 <= hi2)) return false;
  const float dmax = std::fmin(std::fmax(rc.dys, lo2), hi2);
  const float dmin = std::fmin(std::fmax(-rc.dys, lo2), hi2);
  const float tr = std::fmax(ql - (dmax * dmax) * rc.ic, 0.0f);
  const float tl = std::fmax(ql - (dmin * dmin) * rc.ic, 0.0f);
  const float wr = std::sqrt(tr * rc.g), wl = std::sqrt(tl * rc.g);
  const float xr = ((u + rc.sl * dmax) + wr) + k.margin_abs;
  const float xl = ((u + rc.sl * dmin) - wl) - k.margin_abs;
  float f0 = std::floor(xl * 0.0625f), f1 = std::floor(xr * 0.0625f);
  const float r0 = (float)k.rect[0], r1 = (float)(k.rect[2] - 1);
  // the span intersected with the box's columns: empty when it lies wholly to one side
  if (!(f1 >= r0 && f0 <= r1)) return false;
  tx0 = (int)std::fmax(f0, r0);
  tx1 = (int)std::fmin(f1, r1);
  return tx1 >= tx0;
}

void key_prim(const double* mu_d, const double* s_d, const double* q_d, double beta_d, double kappa_d,
              const Cam& cam, const Par& par, KeyOut& o) {
  float mu[3] = {(float)mu_d[0], (float)mu_d[1], (float)mu_d[2]};
  float s[3] = {(float)s_d[0], (float)s_d[1], (float)s_d[2]};
  float qw = (float)q_d[0], qx = (float)q_d[1], qy = (float)q_d[2], qz = (float)q_d[3];
  float beta = (float)beta_d, kappa = (float)kappa_d;
  float V[12];
  for (int i = 0; i < 12; ++i) V[i] = (float)cam.V[i];
  const float fx = (float)cam.fx, fy = (float)cam.fy, cx = (float)cam.cx, cy = (float)cam.cy;
  const float znear = (float)cam.znear;
  const float rho = (float)par.rho, dil = (float)par.dilation, amin = (float)par.alpha_min;
  const float mrel = (float)par.margin_rel, mabs = (float)par.margin_abs, cfov = (float)par.clamp_fov;

  // camera-space mean
  float tx = ((V[0] * mu[0] + V[1] * mu[1]) + V[2] * mu[2]) + V[3];
  float ty = ((V[4] * mu[0] + V[5] * mu[1]) + V[6] * mu[2]) + V[7];
  float tz = ((V[8] * mu[0] + V[9] * mu[1]) + V[10] * mu[2]) + V[11];
  bool valid = tz > znear;
  float iz = 1.0f / tz;
  float u = fx * (tx * iz) + cx;
  float v = fy * (ty * iz) + cy;

  // rotation from the normalised quaternion (w,x,y,z)
  float n2 = ((qw * qw + qx * qx) + qy * qy) + qz * qz;
  valid = valid && (n2 > 0.0f);
  float rn = 1.0f / std::sqrt(n2);
  float w = qw * rn, x = qx * rn, y = qy * rn, z = qz * rn;
  float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  float wx = w * x, wy = w * y, wz = w * z;
  float R[9];
  R[0] = 1.0f - 2.0f * (yy + zz);
  R[1] = 2.0f * (xy - wz);
  R[2] = 2.0f * (xz + wy);
  R[3] = 2.0f * (xy + wz);
  R[4] = 1.0f - 2.0f * (xx + zz);
  R[5] = 2.0f * (yz - wx);
  R[6] = 2.0f * (xz - wy);
  R[7] = 2.0f * (yz + wx);
  R[8] = 1.0f - 2.0f * (xx + yy);

  // shape modification on the scale vector
  valid = valid && (beta > 0.0f);
  float phi = key_phi(beta, rho, par.phi_mode);
  float sp[3] = {phi * s[0], phi * s[1], phi * s[2]};
  float M[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) M[3 * i + j] = R[3 * i + j] * sp[j];
  float Sg[9];
  for (int i = 0; i < 3; ++i)
    for (int j = i; j < 3; ++j) {
      float t = (M[3 * i + 0] * M[3 * j + 0] + M[3 * i + 1] * M[3 * j + 1]) + M[3 * i + 2] * M[3 * j + 2];
      Sg[3 * i + j] = t;
      Sg[3 * j + i] = t;
    }

  // perspective Jacobian with the tangent clamp
  float limx = (cfov * (0.5f * (float)cam.W)) / fx;
  float limy = (cfov * (0.5f * (float)cam.H)) / fy;
  float rx = tx * iz;
  rx = std::fmin(std::fmax(rx, -limx), limx);
  float txc = rx * tz;
  float ry = ty * iz;
  ry = std::fmin(std::fmax(ry, -limy), limy);
  float tyc = ry * tz;
  float iz2 = iz * iz;
  float J00 = fx * iz, J02 = -((fx * txc) * iz2);
  float J11 = fy * iz, J12 = -((fy * tyc) * iz2);
  float T[6];
  for (int j = 0; j < 3; ++j) {
    T[j] = J00 * V[j] + J02 * V[8 + j];
    T[3 + j] = J11 * V[4 + j] + J12 * V[8 + j];
  }
  float U[6];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j)
      U[3 * i + j] = (T[3 * i + 0] * Sg[0 + j] + T[3 * i + 1] * Sg[3 + j]) + T[3 * i + 2] * Sg[6 + j];
  float S00 = (U[0] * T[0] + U[1] * T[1]) + U[2] * T[2];
  float S01 = (U[0] * T[3] + U[1] * T[4]) + U[2] * T[5];
  float S11 = (U[3] * T[3] + U[4] * T[4]) + U[5] * T[5];
  float a = S00 + dil, b = S01, c = S11 + dil;
  float det = a * c - b * b;
  valid = valid && (det > 0.0f);

  // opacity-aware, beta-dependent extent: alpha = kappa * G >= alpha_min  <=>  q <= q*
  float ratio = kappa / amin;
  valid = valid && (ratio > 1.0f);
  const float ln2 = (float)std::log(2.0);
  float L = key_log2(ratio) * ln2;
  float a2 = 2.0f * L;
  float qs;
  if (par.mode == 0) {
    float e2 = (2.0f / beta) * key_log2(a2);
    qs = key_exp2(e2);
  } else {
    qs = a2;
  }
  float onep = 1.0f + mrel;
  float hx = std::sqrt(qs * a), hy = std::sqrt(qs * c);
  hx = hx * onep + mabs;
  hy = hy * onep + mabs;
  hx = std::fmin(hx, 1.0e7f);
  hy = std::fmin(hy, 1.0e7f);
  const int tiles_x = (cam.W + TILE - 1) / TILE, tiles_y = (cam.H + TILE - 1) / TILE;
  float fx0 = std::floor((u - hx) / 16.0f);
  float fx1 = std::floor((u + hx) / 16.0f) + 1.0f;
  float fy0 = std::floor((v - hy) / 16.0f);
  float fy1 = std::floor((v + hy) / 16.0f) + 1.0f;
  fx0 = std::fmin(std::fmax(fx0, 0.0f), (float)tiles_x);
  fx1 = std::fmin(std::fmax(fx1, 0.0f), (float)tiles_x);
  fy0 = std::fmin(std::fmax(fy0, 0.0f), (float)tiles_y);
  fy1 = std::fmin(std::fmax(fy1, 0.0f), (float)tiles_y);
  int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
  o.mean2d[0] = u; o.mean2d[1] = v;
  o.cov2d[0] = a; o.cov2d[1] = b; o.cov2d[2] = c;
  o.qstar = qs;
  o.qlim = (qs * onep) * onep;
  o.margin_abs = mabs;
  o.rect[0] = x0; o.rect[1] = y0; o.rect[2] = x1; o.rect[3] = y1;
  uint32_t touched = 0;
  if (valid && x1 > x0 && y1 > y0) {
    const RowConsts rc = row_consts(o);
    for (int ty = y0; ty < y1; ++ty) {
      int t0, t1;
      if (row_span(o, rc, ty, t0, t1)) touched += (uint32_t)(t1 - t0 + 1);
    }
  }
  uint32_t zb;
  std::memcpy(&zb, &tz, 4);
  o.depth_key = touched ? zb : 0xffffffffu;
  if (!touched) o.rect[0] = o.rect[1] = o.rect[2] = o.rect[3] = 0;
  o.touched = touched;
}

// ---------------------------------------------------------------------------
// 2. FP64 projection, generic in the scalar type.
// ---------------------------------------------------------------------------
template <int K>
struct Dual {
  double v;
  double d[K];
  Dual() : v(0) { for (int i = 0; i < K; ++i) d[i] = 0; }
  Dual(double x) : v(x) { for (int i = 0; i < K; ++i) d[i] = 0; }
};
template <int K> Dual<K> operator+(const Dual<K>& a, const Dual<K>& b) { Dual<K> r; r.v = a.v + b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] + b.d[i]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a, const Dual<K>& b) { Dual<K> r; r.v = a.v - b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] - b.d[i]; return r; }
template <int K> Dual<K> operator-(const Dual<K>& a) { Dual<K> r; r.v = -a.v; for (int i = 0; i < K; ++i) r.d[i] = -a.d[i]; return r; }
template <int K> Dual<K> operator*(const Dual<K>& a, const Dual<K>& b) { Dual<K> r; r.v = a.v * b.v; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b.v + a.v * b.d[i]; return r; }
template <int K> Dual<K> operator/(const Dual<K>& a, const Dual<K>& b) { Dual<K> r; r.v = a.v / b.v; for (int i = 0; i < K; ++i) r.d[i] = (a.d[i] * b.v - a.v * b.d[i]) / (b.v * b.v); return r; }
template <int K> Dual<K> operator+(const Dual<K>& a, double b) { return a + Dual<K>(b); }
template <int K> Dual<K> operator+(double a, const Dual<K>& b) { return Dual<K>(a) + b; }
template <int K> Dual<K> operator-(const Dual<K>& a, double b) { return a - Dual<K>(b); }
template <int K> Dual<K> operator-(double a, const Dual<K>& b) { return Dual<K>(a) - b; }
template <int K> Dual<K> operator*(const Dual<K>& a, double b) { Dual<K> r; r.v = a.v * b; for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * b; return r; }
template <int K> Dual<K> operator*(double a, const Dual<K>& b) { return b * a; }
template <int K> Dual<K> operator/(const Dual<K>& a, double b) { return a * (1.0 / b); }
template <int K> Dual<K> operator/(double a, const Dual<K>& b) { return Dual<K>(a) / b; }
template <int K> Dual<K> dsqrt(const Dual<K>& a) { Dual<K> r; r.v = std::sqrt(a.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] / (2.0 * r.v); return r; }
template <int K> Dual<K> dexp(const Dual<K>& a) { Dual<K> r; r.v = std::exp(a.v); for (int i = 0; i < K; ++i) r.d[i] = a.d[i] * r.v; return r; }
template <int K> double val(const Dual<K>& a) { return a.v; }
inline double dsqrt(double a) { return std::sqrt(a); }
inline double dexp(double a) { return std::exp(a); }
inline double val(double a) { return a; }

// psi(x) = d ln Gamma(x) / dx for x > 0: psi(x) = psi(x + 1) - 1/x until x >= 10, then the
// asymptotic series ln x - 1/(2x) - sum_k B_2k / (2k x^2k) with Bernoulli numbers B_2 .. B_12
// (1/6, -1/30, 1/42, -1/30, 5/66, -691/2730); the first omitted term is below 1e-16 at x >= 10.
double digamma(double x) {
  double acc = 0.0;
  for (int k = 0; k < 16 && x < 10.0; ++k) {
    acc -= 1.0 / x;
    x += 1.0;
  }
  double r2 = 1.0 / (x * x);
  double s = r2 * (1.0 / 12 - r2 * (1.0 / 120 - r2 * (1.0 / 252 - r2 * (1.0 / 240 - r2 * (1.0 / 132 - r2 * 691.0 / 32760)))));
  return acc + std::log(x) - 0.5 / x - s;
}

// The scale modification phi(beta) (its value and, for dual numbers, its derivative):
//   phi_mode 0: phi_bar_rho(beta) = 2 / (1 + exp(-(rho beta - 2 rho)))                 Eq. approx
//   phi_mode 1: phi_n(beta) = 2 Gamma(3/beta) / Gamma(1/beta)   (Eq. probablity, normalised so that
//               phi_n(2) = 1 like phi_bar); d ln phi_n / d beta = (psi(1/beta) - 3 psi(3/beta)) / beta^2
//   phi_mode 2: sqrt(phi_n(beta)) (phi_n read as a variance ratio, Eq. effective)
inline double phi_n_log(double b) { return std::lgamma(3.0 / b) - std::lgamma(1.0 / b) + std::log(2.0); }
inline double phi_mod(double beta, const Par& par) {
  if (par.phi_mode == 0) return 2.0 / (1.0 + std::exp(-(par.rho * beta - 2.0 * par.rho)));
  return std::exp((par.phi_mode == 2 ? 0.5 : 1.0) * phi_n_log(beta));
}
template <int K> Dual<K> phi_mod(const Dual<K>& beta, const Par& par) {
  if (par.phi_mode == 0) return 2.0 / (1.0 + dexp(-(par.rho * beta - 2.0 * par.rho)));
  const double c = par.phi_mode == 2 ? 0.5 : 1.0, b = beta.v;
  Dual<K> r;
  r.v = std::exp(c * phi_n_log(b));
  const double slope = c * r.v * (digamma(1.0 / b) - 3.0 * digamma(3.0 / b)) / (b * b);
  for (int i = 0; i < K; ++i) r.d[i] = slope * beta.d[i];
  return r;
}

// clamp(x, lo, hi) as a function of x: constant (zero derivative) when clamped
template <class S> S clampv(const S& x, double lo, double hi) {
  if (val(x) < lo) return S(lo);
  if (val(x) > hi) return S(hi);
  return x;
}
template <class S> S relu(const S& x) { return val(x) > 0.0 ? x : S(0.0); }

// Real spherical harmonics: Y_lm = sqrt2 K_lm (-1)^m Q_l^m(z) Re/Im((x+iy)^|m|), Q_l^m = d^m P_l / dz^m,
// K_lm = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!).  Order: l-major, m = -l..l.  (Condon-Shortley phase included.)
double factorial(int n) { double f = 1; for (int i = 2; i <= n; ++i) f *= i; return f; }

template <class S>
void sh_basis(int deg, const S& x, const S& y, const S& z, S* out) {
  const double pi = std::acos(-1.0);
  S cm[4], sm[4];
  cm[0] = S(1.0); sm[0] = S(0.0);
  for (int m = 1; m <= deg; ++m) {
    cm[m] = cm[m - 1] * x - sm[m - 1] * y;
    sm[m] = cm[m - 1] * y + sm[m - 1] * x;
  }
  for (int m = 0; m <= deg; ++m) {
    // Q_l^m for l = m..deg
    S Q[4];
    double dfact = 1.0;
    for (int k = 1; k <= 2 * m - 1; k += 2) dfact *= k;
    Q[m] = S(dfact);
    if (m + 1 <= deg) Q[m + 1] = (double)(2 * m + 1) * z * Q[m];
    for (int l = m + 2; l <= deg; ++l)
      Q[l] = ((double)(2 * l - 1) * z * Q[l - 1] - (double)(l + m - 1) * Q[l - 2]) / (double)(l - m);
    for (int l = m; l <= deg; ++l) {
      double K = std::sqrt((2.0 * l + 1.0) / (4.0 * pi) * factorial(l - m) / factorial(l + m));
      if (m == 0) {
        out[l * l + l] = K * Q[l];
      } else {
        double sgn = (m % 2) ? -1.0 : 1.0;
        double c = std::sqrt(2.0) * K * sgn;
        out[l * l + l + m] = c * Q[l] * cm[m];
        out[l * l + l - m] = c * Q[l] * sm[m];
      }
    }
  }
}

template <class S>
struct Proj {
  S mx, my;      // 2D mean (pixels)
  S ca, cb, cc;  // conic: q = ca dx^2 + 2 cb dx dy + cc dy^2
  S s00, s01, s11;  // 2D covariance incl. dilation
  S raw[3];      // SH colour before the clamp at 0 (SH part only; coefficients enter linearly)
  S hb;          // exponent beta/2 (GEF) or 1 (Gaussian form)
  S kappa;
};

// mu, s, q, beta, kappa as scalars S; shs as plain doubles (they enter linearly, handled outside)
template <class S>
void project(const S mu[3], const S s[3], const S q[4], const S& beta, const S& kappa,
             const double* sh, int deg, const Cam& cam, const Par& par, Proj<S>& o, S* basis_out) {
  const double* V = cam.V;
  S t[3];
  for (int i = 0; i < 3; ++i) t[i] = V[4 * i + 0] * mu[0] + V[4 * i + 1] * mu[1] + V[4 * i + 2] * mu[2] + V[4 * i + 3];
  o.mx = cam.fx * t[0] / t[2] + cam.cx;
  o.my = cam.fy * t[1] / t[2] + cam.cy;

  S nrm = dsqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  S w = q[0] / nrm, x = q[1] / nrm, y = q[2] / nrm, z = q[3] / nrm;
  S R[9];
  R[0] = 1.0 - 2.0 * (y * y + z * z); R[1] = 2.0 * (x * y - w * z); R[2] = 2.0 * (x * z + w * y);
  R[3] = 2.0 * (x * y + w * z); R[4] = 1.0 - 2.0 * (x * x + z * z); R[5] = 2.0 * (y * z - w * x);
  R[6] = 2.0 * (x * z - w * y); R[7] = 2.0 * (y * z + w * x); R[8] = 1.0 - 2.0 * (x * x + y * y);

  // the scale modification (phi_bar_rho by default, Eq. approx), applied to the scale vector
  S phi = phi_mod(beta, par);
  S sp[3] = {phi * s[0], phi * s[1], phi * s[2]};
  S Sig[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      S acc(0.0);
      for (int k = 0; k < 3; ++k) acc = acc + R[3 * i + k] * sp[k] * sp[k] * R[3 * j + k];
      Sig[3 * i + j] = acc;
    }

  // EWA: Sigma' = J W Sigma W^T J^T, W = rotation of the view matrix, J = perspective Jacobian at t
  double limx = par.clamp_fov * 0.5 * cam.W / cam.fx;
  double limy = par.clamp_fov * 0.5 * cam.H / cam.fy;
  S txc = clampv(t[0] / t[2], -limx, limx) * t[2];
  S tyc = clampv(t[1] / t[2], -limy, limy) * t[2];
  S J[6];
  J[0] = cam.fx / t[2]; J[1] = S(0.0); J[2] = -(cam.fx * txc) / (t[2] * t[2]);
  J[3] = S(0.0); J[4] = cam.fy / t[2]; J[5] = -(cam.fy * tyc) / (t[2] * t[2]);
  S Tm[6];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 3; ++j) {
      S acc(0.0);
      for (int k = 0; k < 3; ++k) acc = acc + J[3 * i + k] * V[4 * k + j];
      Tm[3 * i + j] = acc;
    }
  S C2[4];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      S acc(0.0);
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) acc = acc + Tm[3 * i + k] * Sig[3 * k + l] * Tm[3 * j + l];
      C2[2 * i + j] = acc;
    }
  o.s00 = C2[0] + par.dilation;
  o.s01 = C2[1];
  o.s11 = C2[3] + par.dilation;
  S det = o.s00 * o.s11 - o.s01 * o.s01;
  o.ca = o.s11 / det;
  o.cb = -o.s01 / det;
  o.cc = o.s00 / det;

  // SH colour: direction from the camera centre to the mean
  S dv[3] = {mu[0] - cam.campos[0], mu[1] - cam.campos[1], mu[2] - cam.campos[2]};
  S dn = dsqrt(dv[0] * dv[0] + dv[1] * dv[1] + dv[2] * dv[2]);
  S basis[16];
  sh_basis(deg, dv[0] / dn, dv[1] / dn, dv[2] / dn, basis);
  int nb = (deg + 1) * (deg + 1);
  for (int ch = 0; ch < 3; ++ch) {
    S acc(0.5);
    for (int k = 0; k < nb; ++k) acc = acc + basis[k] * sh[3 * k + ch];
    o.raw[ch] = acc;
  }
  if (basis_out)
    for (int k = 0; k < nb; ++k) basis_out[k] = basis[k];
  o.hb = (par.mode == 0) ? beta * 0.5 : S(1.0);
  o.kappa = kappa;
}

// ---------------------------------------------------------------------------
// scene bookkeeping shared by the renderers
// ---------------------------------------------------------------------------
struct SceneIn {
  int64_t n;
  const double *means, *scales, *quats, *betas, *opac, *shs;
  int deg;
};

struct Prepared {
  std::vector<KeyOut> keys;
  std::vector<int64_t> order;     // visible primitives in (depth_key, index) order
  std::vector<Proj<double>> proj; // FP64 projection (valid for visible ones)
  std::vector<double> rgb;        // clamped colour [n,3]
};

void prepare(const SceneIn& sc, const Cam& cam, const Par& par, Prepared& P) {
  int64_t n = sc.n;
  P.keys.resize(n);
  P.proj.resize(n);
  P.rgb.assign(3 * n, 0.0);
  int nb = (sc.deg + 1) * (sc.deg + 1);
  for (int64_t i = 0; i < n; ++i) {
    key_prim(sc.means + 3 * i, sc.scales + 3 * i, sc.quats + 4 * i, sc.betas[i], sc.opac[i], cam, par, P.keys[i]);
    if (!P.keys[i].touched) continue;
    project<double>(sc.means + 3 * i, sc.scales + 3 * i, sc.quats + 4 * i, sc.betas[i], sc.opac[i],
                    sc.shs + 3 * nb * i, sc.deg, cam, par, P.proj[i], nullptr);
    for (int ch = 0; ch < 3; ++ch) P.rgb[3 * i + ch] = std::max(0.0, P.proj[i].raw[ch]);
  }
  P.order.clear();
  for (int64_t i = 0; i < n; ++i)
    if (P.keys[i].touched) P.order.push_back(i);
  std::stable_sort(P.order.begin(), P.order.end(),
                   [&](int64_t a, int64_t b) { return P.keys[a].depth_key < P.keys[b].depth_key; });
}

// per-fragment FP64 evaluation; returns alpha before the skip test and fills G, q, p
inline double frag_alpha(const Proj<double>& pr, double px, double py, int mode, double alpha_max,
                         double& G, double& q, double& p, double& dx, double& dy, bool& clamped) {
  dx = px - pr.mx;
  dy = py - pr.my;
  q = pr.ca * dx * dx + 2.0 * pr.cb * dx * dy + pr.cc * dy * dy;
  if (q < 0.0) q = 0.0;  // conic is positive definite; guards rounding only
  p = (mode == 0) ? std::pow(q, pr.hb) : q;
  G = std::exp(-0.5 * p);
  double a = pr.kappa * G;
  clamped = a > alpha_max;
  return clamped ? alpha_max : a;
}

struct PixOut {
  double C[3];
  double T;
  int32_t ncontrib;
  uint8_t flag;
};

// composite one pixel over a list of primitive indices (already in depth order)
template <class It>
void composite_pixel(It begin, It end, const Prepared& P, const Cam& cam, const Par& par, int px_i, int py_i, PixOut& out) {
  double px = px_i + 0.5, py = py_i + 0.5;
  double T = 1.0, C[3] = {0, 0, 0};
  int32_t nc = 0;
  uint8_t flag = 0;
  for (It it = begin; it != end; ++it) {
    int64_t i = *it;
    const Proj<double>& pr = P.proj[i];
    double G, q, p, dx, dy;
    bool cl;
    double raw = 0;
    double a = frag_alpha(pr, px, py, par.mode, par.alpha_max, G, q, p, dx, dy, cl);
    raw = pr.kappa * G;
    if (std::fabs(raw - par.alpha_min) <= par.flag_tol_alpha * par.alpha_min) flag |= 1;
    if (std::fabs(raw - par.alpha_max) <= par.flag_tol_alpha * par.alpha_max) flag |= 2;
    if (a < par.alpha_min) continue;
    double Tn = T * (1.0 - a);
    if (std::fabs(Tn - par.t_min) <= par.flag_tol_t * par.t_min) flag |= 4;
    if (Tn < par.t_min) break;
    for (int ch = 0; ch < 3; ++ch) C[ch] += P.rgb[3 * i + ch] * a * T;
    T = Tn;
    ++nc;
  }
  for (int ch = 0; ch < 3; ++ch) out.C[ch] = C[ch] + T * cam.bg[ch];
  out.T = T;
  out.ncontrib = nc;
  out.flag = flag;
}

template <class F>
void parallel_for(int64_t n, int nthreads, F&& fn) {
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());
  if (nthreads == 1 || n < 64) {
    for (int64_t i = 0; i < n; ++i) fn(i, 0);
    return;
  }
  std::atomic<int64_t> next(0);
  const int64_t chunk = 16;
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&, t]() {
      for (;;) {
        int64_t s = next.fetch_add(chunk);
        if (s >= n) break;
        int64_t e = std::min(n, s + chunk);
        for (int64_t i = s; i < e; ++i) fn(i, t);
      }
    });
  for (auto& x : th) x.join();
}

SceneIn scene_in(int64_t n, const double* means, const double* scales, const double* quats, const double* betas,
                 const double* opac, const double* shs, int deg) {
  SceneIn s;
  s.n = n; s.means = means; s.scales = scales; s.quats = quats; s.betas = betas; s.opac = opac; s.shs = shs; s.deg = deg;
  return s;
}

// tile lists (for the tiled self-check): per tile, visible primitives in depth order
void tile_lists(const Prepared& P, const Cam& cam, std::vector<std::vector<int64_t>>& lists) {
  int tx = (cam.W + TILE - 1) / TILE, ty = (cam.H + TILE - 1) / TILE;
  lists.assign((size_t)tx * ty, {});
  for (int64_t i : P.order) {
    const KeyOut& k = P.keys[i];
    const RowConsts rc = row_consts(k);
    for (int y = k.rect[1]; y < k.rect[3]; ++y) {
      int t0, t1;
      if (!row_span(k, rc, y, t0, t1)) continue;
      for (int x = t0; x <= t1; ++x) lists[(size_t)y * tx + x].push_back(i);
    }
  }
}

}  // namespace

extern "C" {

int ora_abi_version() { return 1; }

float ora_key_exp2(float x) { return key_exp2(x); }
float ora_key_log2(float x) { return key_log2(x); }

// phi_bar_rho(beta) (Eq. approx) in FP64
void ora_phi_bar(int64_t n, const double* beta, double rho, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = 2.0 / (1.0 + std::exp(-(rho * beta[i] - 2.0 * rho)));
}
// exact modification Gamma(3/beta)/Gamma(1/beta) (Eq. probablity), not normalised
void ora_phi_exact(int64_t n, const double* beta, double* out) {
  for (int64_t i = 0; i < n; ++i) out[i] = std::tgamma(3.0 / beta[i]) / std::tgamma(1.0 / beta[i]);
}
// the modification the projection applies, and its derivative in beta (dual numbers)
void ora_phi_mod(int64_t n, const double* beta, const double* par_d, double* phi, double* dphi) {
  Par par = read_par(par_d);
  for (int64_t i = 0; i < n; ++i) {
    Dual<1> b(beta[i]);
    b.d[0] = 1.0;
    Dual<1> r = phi_mod(b, par);
    phi[i] = r.v;
    dphi[i] = r.d[0];
  }
}
double ora_digamma(double x) { return digamma(x); }
float ora_key_lgamma(float x) { return key_lgamma(x); }
float ora_key_phi(float beta, float rho, int phi_mode) { return key_phi(beta, rho, phi_mode); }

void ora_sh_basis(int deg, int64_t n, const double* dirs, double* out) {
  int nb = (deg + 1) * (deg + 1);
  for (int64_t i = 0; i < n; ++i) {
    double b[16];
    sh_basis<double>(deg, dirs[3 * i], dirs[3 * i + 1], dirs[3 * i + 2], b);
    for (int k = 0; k < nb; ++k) out[nb * i + k] = b[k];
  }
}

// Key module over a scene.  Outputs per primitive: depth key, tile rect, tiles touched,
// and the FP32 2D mean / 2D covariance / q* it used.
void ora_keys(int64_t n, const double* means, const double* scales, const double* quats, const double* betas,
              const double* opac, const double* cam_d, const double* par_d, uint32_t* depth_key, int32_t* rect,
              uint32_t* touched, float* mean2d, float* cov2d, float* qstar) {
  Cam cam = read_cam(cam_d);
  Par par = read_par(par_d);
  for (int64_t i = 0; i < n; ++i) {
    KeyOut k;
    key_prim(means + 3 * i, scales + 3 * i, quats + 4 * i, betas[i], opac[i], cam, par, k);
    depth_key[i] = k.depth_key;
    for (int j = 0; j < 4; ++j) rect[4 * i + j] = k.rect[j];
    touched[i] = k.touched;
    if (mean2d) { mean2d[2 * i] = k.mean2d[0]; mean2d[2 * i + 1] = k.mean2d[1]; }
    if (cov2d) for (int j = 0; j < 3; ++j) cov2d[3 * i + j] = k.cov2d[j];
    if (qstar) qstar[i] = k.qstar;
  }
}

// Sorted (key, value) list: key = tile << 32 | depth_key, value = primitive index, stable in
// primitive index; one entry per tile of each primitive's row spans.  keys/vals hold sum(touched).
void ora_sorted_keys(int64_t n, const double* means, const double* scales, const double* quats, const double* betas,
                     const double* opac, const double* cam_d, const double* par_d, uint64_t* keys, uint32_t* vals) {
  Cam cam = read_cam(cam_d);
  Par par = read_par(par_d);
  const int tiles_x = (cam.W + TILE - 1) / TILE;
  std::vector<std::pair<uint64_t, uint32_t>> kv;
  for (int64_t i = 0; i < n; ++i) {
    KeyOut k;
    key_prim(means + 3 * i, scales + 3 * i, quats + 4 * i, betas[i], opac[i], cam, par, k);
    if (!k.touched) continue;
    const RowConsts rc = row_consts(k);
    for (int y = k.rect[1]; y < k.rect[3]; ++y) {
      int t0, t1;
      if (!row_span(k, rc, y, t0, t1)) continue;
      for (int x = t0; x <= t1; ++x) kv.emplace_back((((uint64_t)y * tiles_x + x) << 32) | k.depth_key, (uint32_t)i);
    }
  }
  std::stable_sort(kv.begin(), kv.end(), [](const auto& a, const auto& b) { return a.first < b.first; });
  for (size_t e = 0; e < kv.size(); ++e) {
    keys[e] = kv[e].first;
    vals[e] = kv[e].second;
  }
}

// FP64 projection per primitive (for pins and preprocess parity).  out[n,12]:
// mx, my, conic a, b, c, cov2d s00, s01, s11, rgb (clamped) r, g, b, visible
void ora_project(int64_t n, const double* means, const double* scales, const double* quats, const double* betas,
                 const double* opac, const double* shs, int deg, const double* cam_d, const double* par_d, double* out) {
  Cam cam = read_cam(cam_d);
  Par par = read_par(par_d);
  int nb = (deg + 1) * (deg + 1);
  for (int64_t i = 0; i < n; ++i) {
    KeyOut k;
    key_prim(means + 3 * i, scales + 3 * i, quats + 4 * i, betas[i], opac[i], cam, par, k);
    Proj<double> p;
    project<double>(means + 3 * i, scales + 3 * i, quats + 4 * i, betas[i], opac[i], shs + 3 * nb * i, deg, cam, par, p, nullptr);
    double* o = out + 12 * i;
    o[0] = p.mx; o[1] = p.my; o[2] = p.ca; o[3] = p.cb; o[4] = p.cc;
    o[5] = p.s00; o[6] = p.s01; o[7] = p.s11;
    for (int ch = 0; ch < 3; ++ch) o[8 + ch] = std::max(0.0, p.raw[ch]);
    o[11] = k.touched ? 1.0 : 0.0;
  }
}

// Render.  pix: linear pixel ids (y*W + x) to evaluate, or null for all W*H pixels
// (then npix must be W*H).  img is [3, npix].  tiled=1 renders from the tile lists.
int ora_render(int64_t n, const double* means, const double* scales, const double* quats, const double* betas,
               const double* opac, const double* shs, int deg, const double* cam_d, const double* par_d, int64_t npix,
               const int64_t* pix, double* img, double* T, int32_t* ncontrib, uint8_t* flags, int tiled, int nthreads) {
  Cam cam = read_cam(cam_d);
  Par par = read_par(par_d);
  SceneIn sc = scene_in(n, means, scales, quats, betas, opac, shs, deg);
  Prepared P;
  prepare(sc, cam, par, P);
  std::vector<std::vector<int64_t>> lists;
  int tx = (cam.W + TILE - 1) / TILE;
  if (tiled) tile_lists(P, cam, lists);
  parallel_for(npix, nthreads, [&](int64_t k, int) {
    int64_t lin = pix ? pix[k] : k;
    int x = (int)(lin % cam.W), y = (int)(lin / cam.W);
    PixOut o;
    if (tiled) {
      const auto& L = lists[(size_t)(y / TILE) * tx + (x / TILE)];
      composite_pixel(L.begin(), L.end(), P, cam, par, x, y, o);
    } else {
      composite_pixel(P.order.begin(), P.order.end(), P, cam, par, x, y, o);
    }
    for (int ch = 0; ch < 3; ++ch) img[ch * npix + k] = o.C[ch];
    if (T) T[k] = o.T;
    if (ncontrib) ncontrib[k] = o.ncontrib;
    if (flags) flags[k] = o.flag;
  });
  return 0;
}

// Analytic FP64 backward of  L = sum_pix sum_ch dL_dimg[ch, pix] * img[ch, pix].
// dL_dimg is [3, npix] over the same pixel list as ora_render.  Outputs (all [n,...], zeroed here):
// g_means[n,3], g_scales[n,3], g_quats[n,4], g_betas[n], g_opac[n], g_shs[n,nb,3];
// inter[n,10] (optional): per-primitive gradients of the 2D quantities
//   (mx, my, conic a, b, c, kappa, hb, r, g, b) -- the compositing stage's output.
// cond (optional, [n, 22 + 3 nb]): the scale of each gradient element's rounding error -- for
// the 2D quantities the sum over pixels of the absolute per-pixel contributions (a sum's
// floating-point error is bounded by a multiple of it), for the parameters the same sums carried
// through the absolute values of the per-primitive Jacobian; per primitive in the order
// inter (10), means (3), scales (3), quats (4), beta, kappa, shs (3 nb).
int ora_backward(int64_t n, const double* means, const double* scales, const double* quats, const double* betas,
                 const double* opac, const double* shs, int deg, const double* cam_d, const double* par_d, int64_t npix,
                 const int64_t* pix, const double* dL, double* g_means, double* g_scales, double* g_quats,
                 double* g_betas, double* g_opac, double* g_shs, double* inter, int nthreads, double* cond) {
  Cam cam = read_cam(cam_d);
  Par par = read_par(par_d);
  SceneIn sc = scene_in(n, means, scales, quats, betas, opac, shs, deg);
  Prepared P;
  prepare(sc, cam, par, P);
  int nb = (deg + 1) * (deg + 1);
  if (nthreads <= 0) nthreads = (int)std::max(1u, std::thread::hardware_concurrency());

  // pixel stage: per thread, a list of (primitive, 10 partials)
  struct Rec { int64_t i; double g[10]; };
  std::vector<std::vector<Rec>> recs(nthreads);
  parallel_for(npix, nthreads, [&](int64_t k, int tid) {
    double gC[3] = {dL[k], dL[npix + k], dL[2 * npix + k]};
    if (gC[0] == 0.0 && gC[1] == 0.0 && gC[2] == 0.0) return;
    int64_t lin = pix ? pix[k] : k;
    int x = (int)(lin % cam.W), y = (int)(lin / cam.W);
    double px = x + 0.5, py = y + 0.5;
    struct Fr { int64_t i; double a, G, q, p, dx, dy, T; bool cl; };
    std::vector<Fr> fr;
    double T = 1.0;
    for (int64_t i : P.order) {
      const Proj<double>& pr = P.proj[i];
      Fr f;
      f.i = i;
      f.a = frag_alpha(pr, px, py, par.mode, par.alpha_max, f.G, f.q, f.p, f.dx, f.dy, f.cl);
      if (f.a < par.alpha_min) continue;
      double Tn = T * (1.0 - f.a);
      if (Tn < par.t_min) break;
      f.T = T;
      fr.push_back(f);
      T = Tn;
    }
    // S = colour composited behind the current fragment (absolute), starting with the background
    double S[3] = {T * cam.bg[0], T * cam.bg[1], T * cam.bg[2]};
    for (int64_t j = (int64_t)fr.size() - 1; j >= 0; --j) {
      const Fr& f = fr[j];
      const Proj<double>& pr = P.proj[f.i];
      const double* c = &P.rgb[3 * f.i];
      Rec r;
      r.i = f.i;
      double dLda = 0.0;
      for (int ch = 0; ch < 3; ++ch) {
        dLda += gC[ch] * (c[ch] * f.T - S[ch] / (1.0 - f.a));
        r.g[7 + ch] = gC[ch] * f.a * f.T;
      }
      for (int ch = 0; ch < 3; ++ch) S[ch] += c[ch] * f.a * f.T;
      double dLdk = 0, dLdG = 0;
      if (!f.cl) {
        dLdk = dLda * f.G;
        dLdG = dLda * pr.kappa;
      }
      double dLdp = dLdG * (-0.5 * f.G);
      double dLdq = 0, dLdhb = 0;
      if (par.mode == 0) {
        if (f.q > 1e-12) {
          dLdq = dLdp * pr.hb * f.p / f.q;
          dLdhb = dLdp * f.p * std::log(f.q);
        }
      } else {
        dLdq = dLdp;
      }
      r.g[0] = dLdq * (-2.0 * (pr.ca * f.dx + pr.cb * f.dy));
      r.g[1] = dLdq * (-2.0 * (pr.cb * f.dx + pr.cc * f.dy));
      r.g[2] = dLdq * f.dx * f.dx;
      r.g[3] = dLdq * 2.0 * f.dx * f.dy;
      r.g[4] = dLdq * f.dy * f.dy;
      r.g[5] = dLdk;
      r.g[6] = dLdhb;
      recs[tid].push_back(r);
    }
  });
  std::vector<double> acc((size_t)n * 10, 0.0), acc_abs(cond ? (size_t)n * 10 : 0, 0.0);
  for (auto& v : recs)
    for (auto& r : v)
      for (int j = 0; j < 10; ++j) {
        acc[(size_t)r.i * 10 + j] += r.g[j];
        if (cond) acc_abs[(size_t)r.i * 10 + j] += std::fabs(r.g[j]);
      }
  if (inter) std::memcpy(inter, acc.data(), sizeof(double) * 10 * n);
  const int64_t ncond = 22 + 3 * nb;
  if (cond) std::memset(cond, 0, sizeof(double) * (size_t)ncond * n);

  std::memset(g_means, 0, sizeof(double) * 3 * n);
  std::memset(g_scales, 0, sizeof(double) * 3 * n);
  std::memset(g_quats, 0, sizeof(double) * 4 * n);
  std::memset(g_betas, 0, sizeof(double) * n);
  std::memset(g_opac, 0, sizeof(double) * n);
  std::memset(g_shs, 0, sizeof(double) * 3 * nb * n);

  // primitive stage: exact Jacobian of the projection by forward-mode dual numbers
  constexpr int ND = 12;  // mu(3) s(3) q(4) beta kappa
  using D = Dual<ND>;
  parallel_for(n, nthreads, [&](int64_t i, int) {
    const double* g = &acc[(size_t)i * 10];
    bool any = false;
    for (int j = 0; j < 10; ++j) any = any || (g[j] != 0.0);
    if (!any || !P.keys[i].touched) return;
    D mu[3], s[3], q[4], beta, kappa;
    for (int j = 0; j < 3; ++j) { mu[j] = D(means[3 * i + j]); mu[j].d[j] = 1.0; }
    for (int j = 0; j < 3; ++j) { s[j] = D(scales[3 * i + j]); s[j].d[3 + j] = 1.0; }
    for (int j = 0; j < 4; ++j) { q[j] = D(quats[4 * i + j]); q[j].d[6 + j] = 1.0; }
    beta = D(betas[i]); beta.d[10] = 1.0;
    kappa = D(opac[i]); kappa.d[11] = 1.0;
    Proj<D> pr;
    D basis[16];
    project<D>(mu, s, q, beta, kappa, shs + 3 * nb * i, deg, cam, par, pr, basis);
    // colour gradient through the clamp at zero
    double graw[3];
    for (int ch = 0; ch < 3; ++ch) graw[ch] = (pr.raw[ch].v > 0.0) ? g[7 + ch] : 0.0;
    const D* outs[10] = {&pr.mx, &pr.my, &pr.ca, &pr.cb, &pr.cc, &pr.kappa, &pr.hb, &pr.raw[0], &pr.raw[1], &pr.raw[2]};
    double gin[10];
    for (int j = 0; j < 7; ++j) gin[j] = g[j];
    for (int ch = 0; ch < 3; ++ch) gin[7 + ch] = graw[ch];
    double gp[ND] = {0};
    for (int o = 0; o < 10; ++o)
      for (int k = 0; k < ND; ++k) gp[k] += gin[o] * outs[o]->d[k];
    for (int j = 0; j < 3; ++j) g_means[3 * i + j] = gp[j];
    for (int j = 0; j < 3; ++j) g_scales[3 * i + j] = gp[3 + j];
    for (int j = 0; j < 4; ++j) g_quats[4 * i + j] = gp[6 + j];
    g_betas[i] = gp[10];
    g_opac[i] = gp[11];
    for (int k = 0; k < nb; ++k)
      for (int ch = 0; ch < 3; ++ch) g_shs[(size_t)3 * nb * i + 3 * k + ch] = basis[k].v * graw[ch];
    if (cond) {
      double* c = cond + (size_t)ncond * i;
      const double* ga = &acc_abs[(size_t)i * 10];
      double gin_abs[10];
      for (int j = 0; j < 7; ++j) gin_abs[j] = ga[j];
      for (int ch = 0; ch < 3; ++ch) gin_abs[7 + ch] = (pr.raw[ch].v > 0.0) ? ga[7 + ch] : 0.0;
      for (int j = 0; j < 10; ++j) c[j] = ga[j];
      for (int k = 0; k < ND; ++k) {
        double t = 0.0;
        for (int o = 0; o < 10; ++o) t += gin_abs[o] * std::fabs(outs[o]->d[k]);
        c[10 + k] = t;
      }
      for (int k = 0; k < nb; ++k)
        for (int ch = 0; ch < 3; ++ch) c[22 + 3 * k + ch] = std::fabs(basis[k].v) * gin_abs[7 + ch];
    }
  });
  return 0;
}

}  // extern "C"
