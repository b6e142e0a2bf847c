// Per-primitive kernels: projection (forward) and its chain rule (backward).
//
// Forward, per primitive (Sec. 4.1, Sec. 4.2):
//   phi_bar_rho(beta) = 2 / (1 + exp(-rho (beta - 2)))            Eq. approx (App. B.2: rho = 0.1)
//   or phi_n(beta) = 2 Gamma(3/beta) / Gamma(1/beta) (or its root)   Eq. probablity, normalised
//   Sigma = R diag(phi_bar s)^2 R^T                                  Sec. 4.1 (scale vector modified by phi)
//   Sigma' = J W Sigma W^T J^T + dilation I, conic = Sigma'^-1       Sec. 4.1 (EWA, Zwicker et al.)
//   extent: alpha = kappa exp(-1/2 q^(beta/2)) >= alpha_min  <=>  q <= q* = (2 ln(kappa/alpha_min))^(2/beta)
//   colour = max(0, sum_lm c_lm Y_lm(dir) + 1/2)                     Sec. 4.1 (SH as in Gaussian splatting)
// Everything that decides an integer (visibility, depth key, tile rectangle) runs on the
// fixed-order FP32 key path of common.cuh; the SH colour uses ordinary FP32 arithmetic.
#include "common.cuh"
#include "kernels.cuh"
#include "keypath.cuh"

namespace ges {

namespace {

// Real SH basis of degree <= DEG at unit direction (x,y,z): Y[0..(DEG+1)^2).
template <int DEG>
__device__ __forceinline__ void sh_eval(float x, float y, float z, float* Y) {
  Y[0] = (float)sh_norm(0, 0);
  if (DEG < 1) return;
  const float n11 = (float)sh_norm(1, 1), n10 = (float)sh_norm(1, 0);
  Y[1] = -n11 * y;
  Y[2] = n10 * z;
  Y[3] = -n11 * x;
  if (DEG < 2) return;
  const float n22 = (float)sh_norm(2, 2), n21 = (float)sh_norm(2, 1), n20 = (float)sh_norm(2, 0);
  const float xx = x * x, yy = y * y, zz = z * z;
  Y[4] = 6.0f * n22 * x * y;
  Y[5] = -3.0f * n21 * y * z;
  Y[6] = 0.5f * n20 * (3.0f * zz - 1.0f);
  Y[7] = -3.0f * n21 * x * z;
  Y[8] = 3.0f * n22 * (xx - yy);
  if (DEG < 3) return;
  const float n33 = (float)sh_norm(3, 3), n32 = (float)sh_norm(3, 2), n31 = (float)sh_norm(3, 1),
              n30 = (float)sh_norm(3, 0);
  Y[9] = -15.0f * n33 * y * (3.0f * xx - yy);
  Y[10] = 30.0f * n32 * x * y * z;
  Y[11] = -1.5f * n31 * y * (5.0f * zz - 1.0f);
  Y[12] = 0.5f * n30 * z * (5.0f * zz - 3.0f);
  Y[13] = -1.5f * n31 * x * (5.0f * zz - 1.0f);
  Y[14] = 15.0f * n32 * z * (xx - yy);
  Y[15] = -15.0f * n33 * x * (xx - 3.0f * yy);
}

// Gradient of each basis polynomial with respect to (x,y,z) (the radial part is removed by the caller).
template <int DEG>
__device__ __forceinline__ void sh_grad(float x, float y, float z, float3* dY) {
  dY[0] = make_float3(0.f, 0.f, 0.f);
  if (DEG < 1) return;
  const float n11 = (float)sh_norm(1, 1), n10 = (float)sh_norm(1, 0);
  dY[1] = make_float3(0.f, -n11, 0.f);
  dY[2] = make_float3(0.f, 0.f, n10);
  dY[3] = make_float3(-n11, 0.f, 0.f);
  if (DEG < 2) return;
  const float n22 = (float)sh_norm(2, 2), n21 = (float)sh_norm(2, 1), n20 = (float)sh_norm(2, 0);
  dY[4] = make_float3(6.0f * n22 * y, 6.0f * n22 * x, 0.f);
  dY[5] = make_float3(0.f, -3.0f * n21 * z, -3.0f * n21 * y);
  dY[6] = make_float3(0.f, 0.f, 3.0f * n20 * z);
  dY[7] = make_float3(-3.0f * n21 * z, 0.f, -3.0f * n21 * x);
  dY[8] = make_float3(6.0f * n22 * x, -6.0f * n22 * y, 0.f);
  if (DEG < 3) return;
  const float n33 = (float)sh_norm(3, 3), n32 = (float)sh_norm(3, 2), n31 = (float)sh_norm(3, 1),
              n30 = (float)sh_norm(3, 0);
  const float xx = x * x, yy = y * y, zz = z * z;
  dY[9] = make_float3(-90.0f * n33 * x * y, -45.0f * n33 * (xx - yy), 0.f);
  dY[10] = make_float3(30.0f * n32 * y * z, 30.0f * n32 * x * z, 30.0f * n32 * x * y);
  dY[11] = make_float3(0.f, -1.5f * n31 * (5.0f * zz - 1.0f), -15.0f * n31 * y * z);
  dY[12] = make_float3(0.f, 0.f, 0.5f * n30 * (15.0f * zz - 3.0f));
  dY[13] = make_float3(-1.5f * n31 * (5.0f * zz - 1.0f), 0.f, -15.0f * n31 * x * z);
  dY[14] = make_float3(30.0f * n32 * x * z, -30.0f * n32 * y * z, 15.0f * n32 * (xx - yy));
  dY[15] = make_float3(-45.0f * n33 * (xx - yy), 90.0f * n33 * x * y, 0.f);
}

// coefficients of one primitive: 3 (DEG+1)^2 floats; rows of 48 and 12 floats are 16-byte aligned
template <int DEG>
__device__ __forceinline__ void load_sh(const float* __restrict__ src, float* c) {
  constexpr int kN = 3 * (DEG + 1) * (DEG + 1);
  if constexpr (kN % 4 == 0) {
#pragma unroll
    for (int k = 0; k < kN / 4; ++k) {
      const float4 v = reinterpret_cast<const float4*>(src)[k];
      c[4 * k] = v.x; c[4 * k + 1] = v.y; c[4 * k + 2] = v.z; c[4 * k + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int k = 0; k < kN; ++k) c[k] = src[k];
  }
}

template <int DEG>
__device__ __forceinline__ void store_sh(float* __restrict__ dst, const float* c) {
  constexpr int kN = 3 * (DEG + 1) * (DEG + 1);
  if constexpr (kN % 4 == 0) {
#pragma unroll
    for (int k = 0; k < kN / 4; ++k)
      reinterpret_cast<float4*>(dst)[k] = make_float4(c[4 * k], c[4 * k + 1], c[4 * k + 2], c[4 * k + 3]);
  } else {
#pragma unroll
    for (int k = 0; k < kN; ++k) dst[k] = c[k];
  }
}

// colour = max(0, sum_k c_k Y_k(dir) + 1/2) per channel
template <int DEG>
__device__ __forceinline__ float3 sh_colour(float dx, float dy, float dz, const float* __restrict__ sh) {
  constexpr int kB = (DEG + 1) * (DEG + 1);
  float c[3 * kB];
  load_sh<DEG>(sh, c);
  float Y[kB];
  sh_eval<DEG>(dx, dy, dz, Y);
  float r = 0.5f, g = 0.5f, b = 0.5f;
#pragma unroll
  for (int k = 0; k < kB; ++k) {
    r = fmaf(Y[k], c[3 * k], r);
    g = fmaf(Y[k], c[3 * k + 1], g);
    b = fmaf(Y[k], c[3 * k + 2], b);
  }
  return make_float3(fmaxf(r, 0.f), fmaxf(g, 0.f), fmaxf(b, 0.f));
}

// backward of sh_colour: writes dL/dc (all coefficients) and returns dL/d(dir) (before the
// projection onto the sphere's tangent plane)
template <int DEG>
__device__ __forceinline__ float3 sh_colour_bwd(float dx, float dy, float dz, const float* __restrict__ sh,
                                                const float g_rgb[3], float* __restrict__ gsh) {
  constexpr int kB = (DEG + 1) * (DEG + 1);
  float c[3 * kB];
  load_sh<DEG>(sh, c);
  float Y[kB];
  sh_eval<DEG>(dx, dy, dz, Y);
  float raw[3] = {0.5f, 0.5f, 0.5f};
#pragma unroll
  for (int k = 0; k < kB; ++k) {
    raw[0] = fmaf(Y[k], c[3 * k], raw[0]);
    raw[1] = fmaf(Y[k], c[3 * k + 1], raw[1]);
    raw[2] = fmaf(Y[k], c[3 * k + 2], raw[2]);
  }
  const float gr[3] = {raw[0] > 0.f ? g_rgb[0] : 0.f, raw[1] > 0.f ? g_rgb[1] : 0.f, raw[2] > 0.f ? g_rgb[2] : 0.f};
  float out[3 * kB];
  float3 gd = make_float3(0.f, 0.f, 0.f);
  float3 dY[kB];
  sh_grad<DEG>(dx, dy, dz, dY);
#pragma unroll
  for (int k = 0; k < kB; ++k) {
    out[3 * k] = Y[k] * gr[0];
    out[3 * k + 1] = Y[k] * gr[1];
    out[3 * k + 2] = Y[k] * gr[2];
    if (k > 0) {
      const float gy = c[3 * k] * gr[0] + c[3 * k + 1] * gr[1] + c[3 * k + 2] * gr[2];
      gd.x = fmaf(gy, dY[k].x, gd.x);
      gd.y = fmaf(gy, dY[k].y, gd.y);
      gd.z = fmaf(gy, dY[k].z, gd.z);
    }
  }
  store_sh<DEG>(gsh, out);
  return gd;
}

// psi(x) = d ln Gamma(x) / dx for x > 0 (the backward's slope of the exact modification, ordinary
// FP32): psi(x) = psi(x + 1) - 1/x until x >= 6, then ln x - 1/(2x) - 1/(12 x^2) + 1/(120 x^4) -
// 1/(252 x^6) (the first omitted term, 1/(240 x^8), is below 3e-9 at x >= 6).
__device__ __forceinline__ float digammaf(float x) {
  float acc = 0.0f;
  for (int k = 0; k < 6 && x < 6.0f; ++k) {
    acc -= 1.0f / x;
    x += 1.0f;
  }
  const float r = 1.0f / x, r2 = r * r;
  return acc + logf(x) - 0.5f * r - r2 * ((1.0f / 12.0f) - r2 * ((1.0f / 120.0f) - r2 * (1.0f / 252.0f)));
}

}  // namespace

// ---------------------------------------------------------------------------------------------
// K1: preprocess.  One thread per global primitive id (grid-stride).
// ---------------------------------------------------------------------------------------------
template <class VS>
__global__ void __launch_bounds__(256) k_preprocess(const __grid_constant__ VS vs, const Params P, uint32_t* __restrict__ depth_key,
                                                    uint32_t* __restrict__ sort_keys,
                                                    uint32_t* __restrict__ sort_vals, ushort4* __restrict__ rect,
                                                    Rec* __restrict__ rec, KeyShape* __restrict__ ks,
                                                    uint32_t* __restrict__ tprim) {
  const auto& vt = vs.get();
  const int64_t total = (int64_t)vt.total_prims;
  const unsigned lane = threadIdx.x & 31u;
  // the loop runs warp by warp (the tile count below is warp-cooperative): lanes past the end work
  // on the last primitive and store nothing
  for (int64_t g0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); g0 < total;
       g0 += (int64_t)gridDim.x * blockDim.x) {
    const bool inb = g0 + lane < total;
    const int64_t g = inb ? g0 + lane : total - 1;
    const ViewDesc& vd = vt.v[view_of_prim(vt, g)];
    const int64_t i = g - vd.prim_base;
    const float mx = vd.means[3 * i + 0], my = vd.means[3 * i + 1], mz = vd.means[3 * i + 2];
    const float s0 = vd.scales[3 * i + 0], s1 = vd.scales[3 * i + 1], s2 = vd.scales[3 * i + 2];
    const float4 q4 = *reinterpret_cast<const float4*>(vd.quats + 4 * i);
    const float beta = vd.betas[i], kappa = vd.opac[i];
    const float* V = vd.V;

    // camera-space mean (key path)
    float tx = kadd(kadd(kadd(kmul(V[0], mx), kmul(V[1], my)), kmul(V[2], mz)), V[3]);
    float ty = kadd(kadd(kadd(kmul(V[4], mx), kmul(V[5], my)), kmul(V[6], mz)), V[7]);
    float tz = kadd(kadd(kadd(kmul(V[8], mx), kmul(V[9], my)), kmul(V[10], mz)), V[11]);
    bool valid = tz > vd.znear;
    float iz = kdiv(1.0f, tz);
    float u = kadd(kmul(vd.fx, kmul(tx, iz)), vd.cx);
    float v = kadd(kmul(vd.fy, kmul(ty, iz)), vd.cy);

    // rotation
    float n2 = kadd(kadd(kadd(kmul(q4.x, q4.x), kmul(q4.y, q4.y)), kmul(q4.z, q4.z)), kmul(q4.w, q4.w));
    valid = valid && (n2 > 0.0f);
    float rn = kdiv(1.0f, ksqrt(n2));
    float w = kmul(q4.x, rn), x = kmul(q4.y, rn), y = kmul(q4.z, rn), z = kmul(q4.w, rn);
    float xx = kmul(x, x), yy = kmul(y, y), zz = kmul(z, z), xy = kmul(x, y), xz = kmul(x, z), yz = kmul(y, z);
    float wx = kmul(w, x), wy = kmul(w, y), wz = kmul(w, z);
    float R[9];
    R[0] = ksub(1.0f, kmul(2.0f, kadd(yy, zz)));
    R[1] = kmul(2.0f, ksub(xy, wz));
    R[2] = kmul(2.0f, kadd(xz, wy));
    R[3] = kmul(2.0f, kadd(xy, wz));
    R[4] = ksub(1.0f, kmul(2.0f, kadd(xx, zz)));
    R[5] = kmul(2.0f, ksub(yz, wx));
    R[6] = kmul(2.0f, ksub(xz, wy));
    R[7] = kmul(2.0f, kadd(yz, wx));
    R[8] = ksub(1.0f, kmul(2.0f, kadd(xx, yy)));

    // shape modification on the scale vector
    valid = valid && (beta > 0.0f);
    const float phi = key_phi(beta, P);
    float sp[3] = {kmul(phi, s0), kmul(phi, s1), kmul(phi, s2)};
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) M[3 * a + b] = kmul(R[3 * a + b], sp[b]);
    float Sg[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = a; b < 3; ++b) {
        float t = kadd(kadd(kmul(M[3 * a], M[3 * b]), kmul(M[3 * a + 1], M[3 * b + 1])), kmul(M[3 * a + 2], M[3 * b + 2]));
        Sg[3 * a + b] = t;
        Sg[3 * b + a] = t;
      }

    // EWA Jacobian with the tangent clamp
    float limx = kdiv(kmul(P.clamp_fov, kmul(0.5f, (float)vd.W)), vd.fx);
    float limy = kdiv(kmul(P.clamp_fov, kmul(0.5f, (float)vd.H)), vd.fy);
    float rx = fminf(fmaxf(kmul(tx, iz), -limx), limx);
    float ry = fminf(fmaxf(kmul(ty, iz), -limy), limy);
    float txc = kmul(rx, tz), tyc = kmul(ry, tz);
    float iz2 = kmul(iz, iz);
    float J00 = kmul(vd.fx, iz), J02 = -kmul(kmul(vd.fx, txc), iz2);
    float J11 = kmul(vd.fy, iz), J12 = -kmul(kmul(vd.fy, tyc), iz2);
    float T[6];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T[b] = kadd(kmul(J00, V[b]), kmul(J02, V[8 + b]));
      T[3 + b] = kadd(kmul(J11, V[4 + b]), kmul(J12, V[8 + b]));
    }
    float U[6];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b)
        U[3 * a + b] = kadd(kadd(kmul(T[3 * a], Sg[b]), kmul(T[3 * a + 1], Sg[3 + b])), kmul(T[3 * a + 2], Sg[6 + b]));
    float S00 = kadd(kadd(kmul(U[0], T[0]), kmul(U[1], T[1])), kmul(U[2], T[2]));
    float S01 = kadd(kadd(kmul(U[0], T[3]), kmul(U[1], T[4])), kmul(U[2], T[5]));
    float S11 = kadd(kadd(kmul(U[3], T[3]), kmul(U[4], T[4])), kmul(U[5], T[5]));
    float ca = kadd(S00, P.dilation), cb = S01, cc = kadd(S11, P.dilation);
    float det = ksub(kmul(ca, cc), kmul(cb, cb));
    valid = valid && (det > 0.0f);

    // opacity-aware, beta-dependent extent
    float ratio = kdiv(kappa, P.alpha_min);
    valid = valid && (ratio > 1.0f);
    const float ln2 = (float)0.6931471805599453;
    float L = kmul(key_log2(ratio), ln2);
    float a2 = kmul(2.0f, L);
    float qs;
    if (P.mode == 0) {
      float e2 = kmul(kdiv(2.0f, beta), key_log2(a2));
      qs = key_exp2(e2);
    } else {
      qs = a2;
    }
    float onep = kadd(1.0f, P.margin_rel);
    float hx = kadd(kmul(ksqrt(kmul(qs, ca)), onep), P.margin_abs);
    float hy = kadd(kmul(ksqrt(kmul(qs, cc)), onep), P.margin_abs);
    hx = fminf(hx, 1.0e7f);
    hy = fminf(hy, 1.0e7f);
    float fx0 = floorf(kdiv(ksub(u, hx), 16.0f));
    float fx1 = kadd(floorf(kdiv(kadd(u, hx), 16.0f)), 1.0f);
    float fy0 = floorf(kdiv(ksub(v, hy), 16.0f));
    float fy1 = kadd(floorf(kdiv(kadd(v, hy), 16.0f)), 1.0f);
    fx0 = fminf(fmaxf(fx0, 0.0f), (float)vd.tiles_x);
    fx1 = fminf(fmaxf(fx1, 0.0f), (float)vd.tiles_x);
    fy0 = fminf(fmaxf(fy0, 0.0f), (float)vd.tiles_y);
    fy1 = fminf(fmaxf(fy1, 0.0f), (float)vd.tiles_y);
    int x0 = (int)fx0, x1 = (int)fx1, y0 = (int)fy0, y1 = (int)fy1;
    // list entries: per tile row of the bounding box, the segments its span of the extent meets
    const float ql = kmul(kmul(qs, onep), onep);
    const float4 e4 = make_float4(ca, cb, cc, ql);
    const ushort4 box = make_ushort4((unsigned short)x0, (unsigned short)y0, (unsigned short)x1, (unsigned short)y1);
    const uint32_t h = (inb && valid && x1 > x0 && y1 > y0) ? (uint32_t)(y1 - y0) : 0u;
    const RowSpan rs = make_row_span(e4, u, v, P.margin_abs, box);
    unsigned nslots;
    const unsigned hex = warp_excl_scan(h, nslots);
    uint32_t nentries = 0;
    for (unsigned cb = 0; cb < nslots; cb += 32) {
      const unsigned s = cb + lane;
      const int ow = warp_last_le(hex, s);
      const RowSpan q = shfl_row_span(rs, ow);
      const unsigned qy0 = __shfl_sync(0xffffffffu, (unsigned)y0, ow);
      const unsigned qhex = __shfl_sync(0xffffffffu, hex, ow);
      unsigned w = 0;
      if (s < nslots) {
        int t0, t1;
        if (tile_row_span(q, (int)(qy0 + (s - qhex)), t0, t1))
          w = (unsigned)((t1 >> P.seg_log2) - (t0 >> P.seg_log2) + 1);  // segments the span meets
      }
      unsigned W;
      const unsigned wex = warp_excl_scan(w, W);
      // this lane's primitive owns slots [f, l) of the chunk
      const int f = (int)(hex > cb ? hex : cb) - (int)cb;
      const int l = (int)(hex + h < cb + 32u ? hex + h : cb + 32u) - (int)cb;
      const unsigned a = __shfl_sync(0xffffffffu, wex, f < 31 ? f : 31);
      const unsigned b = __shfl_sync(0xffffffffu, wex + w, l > 0 ? (l - 1 < 31 ? l - 1 : 31) : 0);
      if (h && f < l) nentries += b - a;
    }
    if (!inb) continue;
    const bool touched = nentries > 0;

    const uint32_t dkey = touched ? __float_as_uint(tz) : kCulledKey;
    depth_key[g] = dkey;
    sort_keys[g] = dkey;
    sort_vals[g] = P.id_bits ? ((uint32_t)g | (nentries << P.id_bits)) : (uint32_t)g;
    rect[g] = touched ? box : make_ushort4(0, 0, 0, 0);
    tprim[g] = nentries;
    if (!touched) continue;
    ks[g] = KeyShape{e4, make_float2(u, v), box};

    // SH colour (ordinary FP32)
    float dvx = mx - vd.campos[0], dvy = my - vd.campos[1], dvz = mz - vd.campos[2];
    float dn = rsqrtf(dvx * dvx + dvy * dvy + dvz * dvz);
    const int nb = (vd.sh_degree + 1) * (vd.sh_degree + 1);
    const float* sh = vd.shs + (int64_t)3 * nb * i;
    float3 col;
    switch (vd.sh_degree) {
      case 0: col = sh_colour<0>(dvx * dn, dvy * dn, dvz * dn, sh); break;
      case 1: col = sh_colour<1>(dvx * dn, dvy * dn, dvz * dn, sh); break;
      case 2: col = sh_colour<2>(dvx * dn, dvy * dn, dvz * dn, sh); break;
      default: col = sh_colour<3>(dvx * dn, dvy * dn, dvz * dn, sh); break;
    }
    float idet = 1.0f / det;
    Rec r;
    r.a = make_float4(u, v, ql, P.mode == 0 ? 0.5f * beta : 1.0f);
    r.b = make_float4(cc * idet, -cb * idet, ca * idet, kappa);
    r.c = make_float4(col.x, col.y, col.z, 0.f);
    rec[g] = r;
  }
}

// ---------------------------------------------------------------------------------------------
// K8: preprocess backward.  g2d[3g..3g+2] holds the compositing stage's gradients of
// (mx, my, conic a, conic b) (conic c, kappa, hb, r) (g, b, -, -).  Writes every output.
// ---------------------------------------------------------------------------------------------
template <class VS>
__global__ void __launch_bounds__(256) k_preprocess_bwd(const __grid_constant__ VS vs, const Params P,
                                                        const uint32_t* __restrict__ depth_key,
                                                        const float4* __restrict__ g2d) {
  const auto& vt = vs.get();
  const int64_t total = (int64_t)vt.total_prims;
  for (int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; g < total; g += (int64_t)gridDim.x * blockDim.x) {
    const ViewDesc& vd = vt.v[view_of_prim(vt, g)];
    const int64_t i = g - vd.prim_base;
    const int nb = (vd.sh_degree + 1) * (vd.sh_degree + 1);
    float* gsh = vd.g_shs + (int64_t)3 * nb * i;
    if (depth_key[g] == kCulledKey) {
      for (int k = 0; k < 3; ++k) { vd.g_means[3 * i + k] = 0.f; vd.g_scales[3 * i + k] = 0.f; }
      *reinterpret_cast<float4*>(vd.g_quats + 4 * i) = make_float4(0.f, 0.f, 0.f, 0.f);
      vd.g_betas[i] = 0.f;
      vd.g_opac[i] = 0.f;
      for (int k = 0; k < 3 * nb; ++k) gsh[k] = 0.f;
      continue;
    }
    const float4 ga = g2d[3 * g + 0], gb = g2d[3 * g + 1], gc = g2d[3 * g + 2];
    const float g_mx = ga.x, g_my = ga.y, g_A = ga.z, g_B = ga.w, g_C = gb.x, g_kappa = gb.y, g_hb = gb.z;
    const float g_rgb[3] = {gb.w, gc.x, gc.y};

    const float mu[3] = {vd.means[3 * i], vd.means[3 * i + 1], vd.means[3 * i + 2]};
    const float s[3] = {vd.scales[3 * i], vd.scales[3 * i + 1], vd.scales[3 * i + 2]};
    const float4 q4 = *reinterpret_cast<const float4*>(vd.quats + 4 * i);
    const float beta = vd.betas[i];
    const float* V = vd.V;

    // ---- recompute the forward quantities (ordinary FP32)
    float t[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) t[a] = V[4 * a] * mu[0] + V[4 * a + 1] * mu[1] + V[4 * a + 2] * mu[2] + V[4 * a + 3];
    const float iz = 1.0f / t[2], iz2 = iz * iz;
    const float qn2 = q4.x * q4.x + q4.y * q4.y + q4.z * q4.z + q4.w * q4.w;
    const float rn = rsqrtf(qn2);
    const float w = q4.x * rn, x = q4.y * rn, y = q4.z * rn, z = q4.w * rn;
    float R[9];
    R[0] = 1.f - 2.f * (y * y + z * z); R[1] = 2.f * (x * y - w * z); R[2] = 2.f * (x * z + w * y);
    R[3] = 2.f * (x * y + w * z); R[4] = 1.f - 2.f * (x * x + z * z); R[5] = 2.f * (y * z - w * x);
    R[6] = 2.f * (x * z - w * y); R[7] = 2.f * (y * z + w * x); R[8] = 1.f - 2.f * (x * x + y * y);
    const float phi = P.phi_mode == 0 ? 2.0f / (1.0f + expf(-P.rho * (beta - 2.0f))) : key_phi(beta, P);
    const float sp[3] = {phi * s[0], phi * s[1], phi * s[2]};
    float M[9];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) M[3 * a + b] = R[3 * a + b] * sp[b];
    const float limx = P.clamp_fov * 0.5f * (float)vd.W / vd.fx;
    const float limy = P.clamp_fov * 0.5f * (float)vd.H / vd.fy;
    const float rxr = t[0] * iz, ryr = t[1] * iz;
    const bool clx = rxr < -limx || rxr > limx, cly = ryr < -limy || ryr > limy;
    const float rxc = fminf(fmaxf(rxr, -limx), limx), ryc = fminf(fmaxf(ryr, -limy), limy);
    const float txc = rxc * t[2], tyc = ryc * t[2];
    const float J00 = vd.fx * iz, J02 = -vd.fx * txc * iz2, J11 = vd.fy * iz, J12 = -vd.fy * tyc * iz2;
    float T[6];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      T[b] = J00 * V[b] + J02 * V[8 + b];
      T[3 + b] = J11 * V[4 + b] + J12 * V[8 + b];
    }
    // ---- Sigma' = U U^T + dilation, U = T M (2x3): column b is axis b of the scaled rotation,
    // projected.  The chain below goes through U and W = Q U rather than through the 3x3 gradient
    // of Sigma: for an elongated splat the latter's entries are orders of magnitude larger than
    // the scale gradient along the long axis, which FP32 would then form as a difference of large
    // terms.  With G = [[gA, gB/2], [gB/2, gC]] and dL/dSigma' = -Q G Q:
    //   dL/dM = -2 T^T (Q G W),  dL/dT = -2 (Q G W) M^T,  dL/dsp_b = -(2/sp_b) W_b^T G W_b
    float U[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int b = 0; b < 3; ++b) U[3 * r + b] = T[3 * r] * M[b] + T[3 * r + 1] * M[3 + b] + T[3 * r + 2] * M[6 + b];
    const float ca = U[0] * U[0] + U[1] * U[1] + U[2] * U[2] + P.dilation;
    const float cb = U[0] * U[3] + U[1] * U[4] + U[2] * U[5];
    const float cc = U[3] * U[3] + U[4] * U[4] + U[5] * U[5] + P.dilation;
    const float idet = 1.0f / (ca * cc - cb * cb);
    const float QA = cc * idet, QB = -cb * idet, QC = ca * idet;
    const float h = 0.5f * g_B;
    float Wq[6], Vq[6], QV[6];  // W = Q U, V = G W, QV = Q V
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      Wq[b] = QA * U[b] + QB * U[3 + b];
      Wq[3 + b] = QB * U[b] + QC * U[3 + b];
      Vq[b] = g_A * Wq[b] + h * Wq[3 + b];
      Vq[3 + b] = h * Wq[b] + g_C * Wq[3 + b];
      QV[b] = QA * Vq[b] + QB * Vq[3 + b];
      QV[3 + b] = QB * Vq[b] + QC * Vq[3 + b];
    }
    // dL/dT = -2 QV M^T (2x3)
    float GT[6];
#pragma unroll
    for (int r = 0; r < 2; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c)
        GT[3 * r + c] = -2.f * (QV[3 * r] * M[3 * c] + QV[3 * r + 1] * M[3 * c + 1] + QV[3 * r + 2] * M[3 * c + 2]);
    // ---- T = J W: only J00, J02, J11, J12 are non-zero
    float gJ00 = 0.f, gJ02 = 0.f, gJ11 = 0.f, gJ12 = 0.f;
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      gJ00 += GT[b] * V[b];
      gJ02 += GT[b] * V[8 + b];
      gJ11 += GT[3 + b] * V[4 + b];
      gJ12 += GT[3 + b] * V[8 + b];
    }
    float gt[3] = {0.f, 0.f, 0.f};
    gt[2] += gJ00 * (-vd.fx * iz2) + gJ11 * (-vd.fy * iz2);
    gt[2] += gJ02 * (2.f * vd.fx * txc * iz2 * iz) + gJ12 * (2.f * vd.fy * tyc * iz2 * iz);
    const float gtxc = gJ02 * (-vd.fx * iz2), gtyc = gJ12 * (-vd.fy * iz2);
    if (clx) gt[2] += gtxc * rxc; else gt[0] += gtxc;
    if (cly) gt[2] += gtyc * ryc; else gt[1] += gtyc;
    // ---- 2D mean
    gt[0] += g_mx * vd.fx * iz;
    gt[1] += g_my * vd.fy * iz;
    gt[2] += -(g_mx * vd.fx * t[0] + g_my * vd.fy * t[1]) * iz2;
    float gmu[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) gmu[a] = V[a] * gt[0] + V[4 + a] * gt[1] + V[8 + a] * gt[2];
    // ---- M = R diag(sp): dL/dsp_b from W and V; the rotation through the torques about the body
    // axes, tau_k = dL/dtheta_k for R -> R Rot_k(theta), which is
    //   tau_k = -2 (s_i^2 - s_j^2) (W_i/s_i)^T G (W_j/s_j),  (i, j, k) cyclic,
    // so that a rotation about an axis of equal scales gets an exact zero rather than the
    // difference of two large terms
    float gsp[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) gsp[b] = -2.f * (Wq[b] * Vq[b] + Wq[3 + b] * Vq[3 + b]) / sp[b];
    float tau[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int i = (k + 1) % 3, j = (k + 2) % 3;
      const float wv = Wq[i] * Vq[j] + Wq[3 + i] * Vq[3 + j];
      tau[k] = -2.f * ((sp[i] - sp[j]) * (sp[i] + sp[j]) / (sp[i] * sp[j])) * wv;
    }
    const float gphi = s[0] * gsp[0] + s[1] * gsp[1] + s[2] * gsp[2];
    // d phi / d beta: rho phi (1 - phi/2) for phi_bar; c phi (psi(1/beta) - 3 psi(3/beta)) / beta^2 for
    // phi_n^c (c = 1, or 1/2 for the variance reading)
    float gbeta;
    if (P.phi_mode == 0) {
      gbeta = gphi * P.rho * phi * (1.0f - 0.5f * phi);
    } else {
      const float ib = 1.0f / beta;
      const float dl = (digammaf(ib) - 3.0f * digammaf(3.0f * ib)) * ib * ib;
      gbeta = gphi * phi * (P.phi_mode == 2 ? 0.5f * dl : dl);
    }
    if (P.mode == 0) gbeta += 0.5f * g_hb;
    // ---- quaternion: a body rotation dtheta moves the unit quaternion by q (x) (0, dtheta)/2, whose
    // directions span the tangent space at q orthonormally, so dL/dq = 2 q (x) (0, tau) / |q|
    // (with respect to the unnormalised input, orthogonal to q)
    const float gsc = 2.f * rn;
    const float4 gq = make_float4(-(x * tau[0] + y * tau[1] + z * tau[2]) * gsc,
                                  (w * tau[0] + (y * tau[2] - z * tau[1])) * gsc,
                                  (w * tau[1] + (z * tau[0] - x * tau[2])) * gsc,
                                  (w * tau[2] + (x * tau[1] - y * tau[0])) * gsc);

    // ---- SH colour
    const float dvx = mu[0] - vd.campos[0], dvy = mu[1] - vd.campos[1], dvz = mu[2] - vd.campos[2];
    const float idn = rsqrtf(dvx * dvx + dvy * dvy + dvz * dvz);
    const float dx = dvx * idn, dy = dvy * idn, dz = dvz * idn;
    const float* sh = vd.shs + (int64_t)3 * nb * i;
    float3 gd;
    switch (vd.sh_degree) {
      case 0: gd = sh_colour_bwd<0>(dx, dy, dz, sh, g_rgb, gsh); break;
      case 1: gd = sh_colour_bwd<1>(dx, dy, dz, sh, g_rgb, gsh); break;
      case 2: gd = sh_colour_bwd<2>(dx, dy, dz, sh, g_rgb, gsh); break;
      default: gd = sh_colour_bwd<3>(dx, dy, dz, sh, g_rgb, gsh); break;
    }
    const float dd = dx * gd.x + dy * gd.y + dz * gd.z;
    gmu[0] += (gd.x - dx * dd) * idn;
    gmu[1] += (gd.y - dy * dd) * idn;
    gmu[2] += (gd.z - dz * dd) * idn;

    for (int k = 0; k < 3; ++k) {
      vd.g_means[3 * i + k] = gmu[k];
      vd.g_scales[3 * i + k] = phi * gsp[k];
    }
    *reinterpret_cast<float4*>(vd.g_quats + 4 * i) = gq;
    vd.g_betas[i] = gbeta;
    vd.g_opac[i] = g_kappa;
  }
}

// ---------------------------------------------------------------------------------------------
// launch helpers
// ---------------------------------------------------------------------------------------------
static int grid_for(int64_t total, int num_sms) {
  // grid-stride kernels: enough CTAs for 8 resident 256-thread CTAs per SM, no more than needed
  int64_t need = (total + 255) / 256;
  int64_t cap = (int64_t)num_sms * 8;
  return (int)(need < cap ? (need > 0 ? need : 1) : cap);
}

template <class VS>
void launch_preprocess(const VS& vs, int64_t grid_total, const Params& P, uint32_t* depth_key, uint32_t* sort_keys,
                       uint32_t* sort_vals, ushort4* rect, Rec* rec, KeyShape* ks, uint32_t* tprim, int num_sms,
                       cudaStream_t s) {
  if (grid_total <= 0) return;
  k_preprocess<VS><<<grid_for(grid_total, num_sms), 256, 0, s>>>(vs, P, depth_key, sort_keys, sort_vals, rect, rec, ks,
                                                                  tprim);
  count_launches(1);
}

template <class VS>
void launch_preprocess_bwd(const VS& vs, int64_t grid_total, const Params& P, const uint32_t* depth_key,
                           const float4* g2d, int num_sms, cudaStream_t s) {
  if (grid_total <= 0) return;
  k_preprocess_bwd<VS><<<grid_for(grid_total, num_sms), 256, 0, s>>>(vs, P, depth_key, g2d);
  count_launches(1);
}

// ln2^k / k! rounded to float, computed here in long double and uploaded once per stream use
void set_key_constants(cudaStream_t s) {
  float c[8];
  long double ln2 = 0.693147180559945309417232121458176568L;
  long double t = 1.0L;
  for (int k = 0; k < 8; ++k) {
    if (k > 0) t = t * ln2 / (long double)k;
    c[k] = (float)t;
  }
  cudaMemcpyToSymbolAsync(c_exp2_coef, c, sizeof(c), 0, cudaMemcpyHostToDevice, s);
}

template void launch_preprocess<FrameViews>(const FrameViews&, int64_t, const Params&, uint32_t*, uint32_t*, uint32_t*,
                                            ushort4*, Rec*, KeyShape*, uint32_t*, int, cudaStream_t);
template void launch_preprocess<BatchViews>(const BatchViews&, int64_t, const Params&, uint32_t*, uint32_t*, uint32_t*,
                                            ushort4*, Rec*, KeyShape*, uint32_t*, int, cudaStream_t);
template void launch_preprocess_bwd<FrameViews>(const FrameViews&, int64_t, const Params&, const uint32_t*,
                                                const float4*, int, cudaStream_t);

}  // namespace ges
