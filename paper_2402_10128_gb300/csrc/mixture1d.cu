// The 1D mixture-fitting study (Sec. 3.2; App. A): mixtures of N Gaussians, differences of
// Gaussians (variance ratio nu = 4), Laplacians of Gaussians or generalized exponentials
//   GEF: h(x) = sum_i w_i exp(-|x - mu_i|^beta_i / (2 sigma_i^2 + eps))            (Eq. genmixture)
// fitted to 1D signals by full-batch Adam on the mean squared error, many runs at once; and the
// study's signals (square, triangle, parabolic, half sinusoid, exponential, Gaussian).
//
// One CTA per run, for all epochs: the samples, the residuals, the parameters and the Adam moments
// stay in shared memory.  An epoch is (a) per-component constants, (b) the model at every sample
// and the residual (threads over samples), (c) the gradient: the threads are split into chunks per
// component, each chunk sums its component's partial derivatives times the residual over a stride
// of the samples, and the chunks are added up per parameter, (d) the Adam step (one thread per
// parameter).  Templated on the arithmetic type: float (the study's PyTorch default) or double.
#include <cmath>
#include <cstring>

#include "api_internal.h"

namespace ges {
namespace {

constexpr int kFitThreads = 256;
constexpr int kMaxPoints = 4096;
constexpr int kMaxComponents = 128;

struct FitArgs {
  int32_t n, rows, positive, epochs, n_points;
  int64_t y_stride;
  double lr, b1, b2, adam_eps, nu, mix_eps;
  const void* x;
  const void* y;
  void* params;
  void* loss_hist;
  void* final_loss;
  void* grad;
};

// In float the fits use the hardware's exp2 / log2 and multiply by reciprocals (the study's float
// runs are not reproducible to the last bit anyway); in double they use the library's exp, log,
// pow and true divisions, to follow the FP64 oracle as closely as rounding allows.
template <class T> __device__ __forceinline__ T t_exp(T v);
template <> __device__ __forceinline__ float t_exp<float>(float v) { return exp2f(v * 1.4426950408889634f); }
template <> __device__ __forceinline__ double t_exp<double>(double v) { return exp(v); }
template <class T> __device__ __forceinline__ T t_log(T v);
template <> __device__ __forceinline__ float t_log<float>(float v) { return __log2f(v) * 0.6931471805599453f; }
template <> __device__ __forceinline__ double t_log<double>(double v) { return log(v); }
template <class T> __device__ __forceinline__ T t_pow(T a, T b);  // a >= 0
template <> __device__ __forceinline__ float t_pow<float>(float a, float b) { return exp2f(b * __log2f(a)); }
template <> __device__ __forceinline__ double t_pow<double>(double a, double b) { return pow(a, b); }
// a / b, with ib = 1 / b precomputed: a multiplication in float, the division in double
template <class T> __device__ __forceinline__ T t_div(T a, T b, T ib);
template <> __device__ __forceinline__ float t_div<float>(float a, float, float ib) { return a * ib; }
template <> __device__ __forceinline__ double t_div<double>(double a, double b, double) { return a / b; }
// a / b without a precomputed reciprocal: the fast approximate division in float
template <class T> __device__ __forceinline__ T t_fdiv(T a, T b);
template <> __device__ __forceinline__ float t_fdiv<float>(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double t_fdiv<double>(double a, double b) { return a / b; }
template <class T> __device__ __forceinline__ T t_sqrt(T v);
template <> __device__ __forceinline__ float t_sqrt<float>(float v) { return sqrtf(v); }
template <> __device__ __forceinline__ double t_sqrt<double>(double v) { return sqrt(v); }
template <class T> __device__ __forceinline__ T t_sin(T v);
template <> __device__ __forceinline__ float t_sin<float>(float v) { return sinf(v); }
template <> __device__ __forceinline__ double t_sin<double>(double v) { return sin(v); }
template <class T> __device__ __forceinline__ T t_sign(T v) { return v > T(0) ? T(1) : (v < T(0) ? T(-1) : T(0)); }
template <class T> __device__ __forceinline__ bool t_finite(T v) { return v == v && v - v == T(0); }

template <class T>
struct Comp {  // per-component constants of an epoch
  T w, dw;     // weight and d w / d omega
  T mu, s, beta;
  T D1, D2;    // 2 s^2 + eps; DoG: 2 s^2 / nu + eps
  T iD1, iD2;  // their reciprocals
  T s2, is2, is3;  // s^2, 1 / s^2 and 1 / s^3 (LoG)
  T s4nu;      // 4 s / nu (DoG)
  T nu;
};

// model: 0 Gaussian, 1 DoG, 2 LoG, 3 GEF
template <class T, int M>
__device__ __forceinline__ T comp_value(const Comp<T>& c, T x) {
  const T d = x - c.mu;
  const T d2 = d * d;
  if (M == 0) return c.w * t_exp<T>(-t_div<T>(d2, c.D1, c.iD1));
  if (M == 1) return c.w * (t_exp<T>(-t_div<T>(d2, c.D1, c.iD1)) - t_exp<T>(-t_div<T>(d2, c.D2, c.iD2)));
  if (M == 2) return c.w * ((T(1) - t_div<T>(d2, c.s2, c.is2)) * t_exp<T>(-t_div<T>(d2, c.D1, c.iD1)));
  const T a = d < T(0) ? -d : d;
  return c.w * t_exp<T>(-t_div<T>(t_pow<T>(a, c.beta), c.D1, c.iD1));
}

// adds r * d(component)/d(omega, mu, sigma[, beta]) at x to g[0..rows)
template <class T, int M>
__device__ __forceinline__ void comp_grad(const Comp<T>& c, T x, T r, T* g) {
  const T d = x - c.mu;
  const T d2 = d * d;
  if (M == 0) {
    const T e = t_exp<T>(-t_div<T>(d2, c.D1, c.iD1));
    const T re = r * e;
    g[0] += re * c.dw;
    g[1] += re * c.w * t_div<T>(T(2) * d, c.D1, c.iD1);
    g[2] += re * c.w * t_div<T>(d2 * (T(4) * c.s), c.D1 * c.D1, c.iD1 * c.iD1);
  } else if (M == 1) {
    const T e1 = t_exp<T>(-t_div<T>(d2, c.D1, c.iD1)), e2 = t_exp<T>(-t_div<T>(d2, c.D2, c.iD2));
    g[0] += r * (e1 - e2) * c.dw;
    g[1] += r * c.w * (e1 * t_div<T>(T(2) * d, c.D1, c.iD1) - e2 * t_div<T>(T(2) * d, c.D2, c.iD2));
    g[2] += r * c.w * d2 *
            (e1 * t_div<T>(T(4) * c.s, c.D1 * c.D1, c.iD1 * c.iD1) -
             e2 * t_div<T>(c.s4nu, c.D2 * c.D2, c.iD2 * c.iD2));
  } else if (M == 2) {
    const T e = t_exp<T>(-t_div<T>(d2, c.D1, c.iD1));
    const T u = T(1) - t_div<T>(d2, c.s2, c.is2);
    const T re = r * e;
    g[0] += re * u * c.dw;
    g[1] += re * c.w * (t_div<T>(T(2) * d, c.s2, c.is2) + u * t_div<T>(T(2) * d, c.D1, c.iD1));
    g[2] += re * c.w * d2 *
            (t_div<T>(T(2), c.s2 * c.s, c.is3) + u * t_div<T>(T(4) * c.s, c.D1 * c.D1, c.iD1 * c.iD1));
  } else {
    const T a = d < T(0) ? -d : d;
    const T p = t_pow<T>(a, c.beta);
    const T e = t_exp<T>(-t_div<T>(p, c.D1, c.iD1));
    const T re = r * e;
    g[0] += re * c.dw;
    if (a > T(0)) {  // at a = 0 the mean and shape derivatives are taken as 0 (|.|^beta has no slope there)
      g[1] += re * c.w * t_div<T>(c.beta * t_fdiv<T>(p, a) * t_sign<T>(d), c.D1, c.iD1);
      g[3] += re * c.w * t_div<T>(-p * t_log<T>(a), c.D1, c.iD1);
    }
    g[2] += re * c.w * t_div<T>(p * (T(4) * c.s), c.D1 * c.D1, c.iD1 * c.iD1);
  }
}

template <class T>
struct FitShared {  // carved from dynamic shared memory
  T* x;
  T* y;
  T* r;
  T* p;      // [rows][n]
  T* m;
  T* v;
  T* part;   // [threads][4]
  Comp<T>* c;
  T* red;    // [32]
};

template <class T>
__device__ T block_sum(T v, T* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  T s = T(0);
  if (threadIdx.x < 32) {
    s = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : T(0);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  return red[0];
}

template <class T, int M>
__global__ void __launch_bounds__(kFitThreads) k_fit1d(const __grid_constant__ FitArgs A) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int run = blockIdx.x;
  const int n = A.n, rows = A.rows, S = A.n_points, P = rows * n;
  FitShared<T> sh;
  {
    T* b = reinterpret_cast<T*>(smem);
    sh.x = b;
    sh.y = sh.x + S;
    sh.r = sh.y + S;
    sh.p = sh.r + S;
    sh.m = sh.p + P;
    sh.v = sh.m + P;
    sh.part = sh.v + P;
    sh.red = sh.part + 4 * kFitThreads;
    sh.c = reinterpret_cast<Comp<T>*>(sh.red + 32);
  }
  const T* gx = static_cast<const T*>(A.x);
  const T* gy = static_cast<const T*>(A.y) + (int64_t)run * A.y_stride;
  T* gp = static_cast<T*>(A.params) + (int64_t)run * P;
  for (int s = threadIdx.x; s < S; s += blockDim.x) {
    sh.x[s] = gx[s];
    sh.y[s] = gy[s];
  }
  for (int j = threadIdx.x; j < P; j += blockDim.x) {
    sh.p[j] = gp[j];
    sh.m[j] = T(0);
    sh.v[j] = T(0);
  }
  const int C = kFitThreads / n;  // chunks per component (n <= 128: C >= 2)
  const T inv_S2 = T(2) / T(S);
  const T eps = T(A.mix_eps), nu = T(A.nu), b1 = T(A.b1), b2 = T(A.b2), aeps = T(A.adam_eps);
  T* hist = A.loss_hist ? static_cast<T*>(A.loss_hist) + (int64_t)run * (A.epochs + 1) : nullptr;
  bool dead = false;
  T last_loss = T(0);
  __syncthreads();
  for (int ep = 0; ep <= A.epochs; ++ep) {
    // (a) per-component constants
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      Comp<T> c;
      const T om = sh.p[i];
      c.w = A.positive ? (om < T(0) ? -om : om) : om;
      c.dw = A.positive ? t_sign<T>(om) : T(1);
      c.mu = sh.p[n + i];
      c.s = sh.p[2 * n + i];
      c.beta = rows > 3 ? sh.p[3 * n + i] : T(2);
      c.D1 = T(2) * c.s * c.s + eps;
      c.D2 = T(2) * (c.s * c.s / nu) + eps;
      c.iD1 = T(1) / c.D1;
      c.iD2 = T(1) / c.D2;
      c.s2 = c.s * c.s;
      c.is2 = T(1) / c.s2;
      c.is3 = c.is2 / c.s;
      c.s4nu = T(4) * c.s / nu;
      c.nu = nu;
      sh.c[i] = c;
    }
    __syncthreads();
    // (b) model and residual
    T ls = T(0);
    for (int s = threadIdx.x; s < S; s += blockDim.x) {
      const T xs = sh.x[s];
      T val = T(0);
      for (int i = 0; i < n; ++i) val += comp_value<T, M>(sh.c[i], xs);
      const T r = val - sh.y[s];
      sh.r[s] = r;
      ls += r * r;
    }
    const T loss = block_sum<T>(ls, sh.red) / T(S);
    if (threadIdx.x == 0 && hist) hist[ep] = loss;
    last_loss = loss;
    if (!t_finite<T>(loss)) {
      dead = true;
      if (threadIdx.x == 0 && hist)
        for (int e2 = ep + 1; e2 <= A.epochs; ++e2) hist[e2] = T(NAN);
      break;
    }
    const bool last = ep == A.epochs;
    if (last && !A.grad) break;
    // (c) gradient
    {
      const int t = threadIdx.x;
      T g[4] = {T(0), T(0), T(0), T(0)};
      if (t < n * C) {
        const int i = t / C, ch = t - i * C;
        const Comp<T> c = sh.c[i];
        for (int s = ch; s < S; s += C) comp_grad<T, M>(c, sh.x[s], sh.r[s], g);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) sh.part[4 * t + k] = g[k];
    }
    __syncthreads();
    for (int j = threadIdx.x; j < P; j += blockDim.x) {
      const int k = j / n, i = j - k * n;
      T g = T(0);
      for (int ch = 0; ch < C; ++ch) g += sh.part[4 * (i * C + ch) + k];
      g *= inv_S2;
      if (last) {
        static_cast<T*>(A.grad)[(int64_t)run * P + j] = g;
      } else {
        // (d) Adam, step t = ep + 1: m += (1 - b1)(g - m), v = b2 v + (1 - b2) g^2,
        //     p -= (lr / (1 - b1^t)) m / (sqrt(v) / sqrt(1 - b2^t) + eps)
        const T m = sh.m[j] + (T(1) - b1) * (g - sh.m[j]);
        const T v = b2 * sh.v[j] + (T(1) - b2) * g * g;
        sh.m[j] = m;
        sh.v[j] = v;
        const double c1 = 1.0 - pow(A.b1, (double)(ep + 1));
        const double sc2 = sqrt(1.0 - pow(A.b2, (double)(ep + 1)));
        sh.p[j] -= T(A.lr / c1) * (m / (t_sqrt<T>(v) / T(sc2) + aeps));
      }
    }
    __syncthreads();
  }
  if (dead && A.grad)
    for (int j = threadIdx.x; j < P; j += blockDim.x) static_cast<T*>(A.grad)[(int64_t)run * P + j] = T(NAN);
  for (int j = threadIdx.x; j < P; j += blockDim.x) gp[j] = dead ? T(NAN) : sh.p[j];
  if (threadIdx.x == 0) static_cast<T*>(A.final_loss)[run] = dead ? T(NAN) : last_loss;
}

template <class T>
__global__ void k_signal1d(int kind, T width, int n, T x0, T x1, T* x, T* y) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const T xi = n > 1 ? x0 + (x1 - x0) * T(i) / T(n - 1) : x0;
  const T h = width / T(2);
  const bool inside = xi > -h && xi < h;
  const T a = xi < T(0) ? -xi : xi;
  T v = T(0);
  switch (kind) {
    case 0: v = T(1); break;                                                   // square
    case 1: v = h - a; break;                                                  // triangle
    case 2: v = h * h - xi * xi; break;                                        // parabolic
    case 3: v = t_sin<T>((xi + h) * T(3.14159265358979323846) / width); break;  // half sinusoid
    case 4: v = t_exp<T>(-a); break;                                           // exponential
    default: v = t_exp<T>(-(xi * xi) / (T(2) * width * width)); break;         // Gaussian
  }
  x[i] = xi;
  y[i] = (kind == 5 || inside) ? v : T(0);
}

template <class T>
size_t fit_smem(int S, int P) {
  return sizeof(T) * (3 * (size_t)S + 3 * (size_t)P + 4 * kFitThreads + 32) + sizeof(Comp<T>) * kMaxComponents + 16;
}

template <class T, int M>
cudaError_t launch_fit(const FitArgs& A, int runs, cudaStream_t s) {
  const size_t bytes = fit_smem<T>(A.n_points, A.rows * A.n);
  cudaError_t e = cudaFuncSetAttribute(k_fit1d<T, M>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) return e;
  k_fit1d<T, M><<<runs, kFitThreads, bytes, s>>>(A);
  return cudaGetLastError();
}

template <class T>
cudaError_t launch_fit_model(int model, const FitArgs& A, int runs, cudaStream_t s) {
  switch (model) {
    case 0: return launch_fit<T, 0>(A, runs, s);
    case 1: return launch_fit<T, 1>(A, runs, s);
    case 2: return launch_fit<T, 2>(A, runs, s);
    default: return launch_fit<T, 3>(A, runs, s);
  }
}

}  // namespace
}  // namespace ges

using namespace ges;

extern "C" {

ges_status ges_fit1d_params_default(ges_fit1d_params* out) {
  if (!out) return fail(GES_ERR_INVALID_ARG, "out is NULL");
  out->model = GES_MIX_GEF;
  out->n_components = 5;
  out->positive_weights = 1;
  out->epochs = 1000;
  out->precision = 32;
  out->lr = 0.01;
  out->beta1 = 0.9;
  out->beta2 = 0.999;
  out->adam_eps = 1e-8;
  out->nu = 4.0;
  out->mix_eps = 1e-8;
  return GES_OK;
}

ges_status ges_signal1d(ges_ctx* ctx, int32_t kind, double width, int32_t n_points, double x0, double x1,
                        int32_t precision, void* x, void* y, void* stream) {
  if (!ctx || !x || !y) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  if (kind < GES_SIGNAL_SQUARE || kind > GES_SIGNAL_GAUSSIAN) return fail(GES_ERR_INVALID_ARG, "unknown signal %d", kind);
  if (n_points < 1 || !(width > 0.0) || (precision != 32 && precision != 64))
    return fail(GES_ERR_INVALID_ARG, "need n_points >= 1, width > 0 and precision 32 or 64");
  ges_status st = use_device(ctx->device);
  if (st != GES_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const unsigned grid = (unsigned)((n_points + 255) / 256);
  if (precision == 32)
    k_signal1d<float><<<grid, 256, 0, s>>>(kind, (float)width, n_points, (float)x0, (float)x1, (float*)x, (float*)y);
  else
    k_signal1d<double><<<grid, 256, 0, s>>>(kind, width, n_points, x0, x1, (double*)x, (double*)y);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? GES_OK : cuda_fail(e, "signal launch");
}

ges_status ges_fit1d(ges_ctx* ctx, const ges_fit1d_params* p, int32_t runs, int32_t n_points, const void* x,
                     const void* y, int64_t y_stride, void* params, void* loss_hist, void* final_loss, void* grad,
                     void* stream) {
  if (!ctx || !p || !x || !y || !params || !final_loss) return fail(GES_ERR_INVALID_ARG, "NULL argument");
  if (p->model < GES_MIX_GAUSSIAN || p->model > GES_MIX_GEF) return fail(GES_ERR_INVALID_ARG, "unknown model %d", p->model);
  if (p->n_components < 1 || p->n_components > kMaxComponents)
    return fail(GES_ERR_INVALID_ARG, "n_components must lie in [1, %d]", kMaxComponents);
  if (n_points < 1 || n_points > kMaxPoints) return fail(GES_ERR_INVALID_ARG, "n_points must lie in [1, %d]", kMaxPoints);
  if (runs < 0 || p->epochs < 0 || y_stride < 0) return fail(GES_ERR_INVALID_ARG, "runs, epochs and y_stride must be >= 0");
  if (p->precision != 32 && p->precision != 64) return fail(GES_ERR_INVALID_ARG, "precision must be 32 or 64");
  if (!(p->lr > 0.0) || !(p->beta1 >= 0.0 && p->beta1 < 1.0) || !(p->beta2 >= 0.0 && p->beta2 < 1.0) ||
      !(p->adam_eps >= 0.0) || !(p->nu > 0.0) || !(p->mix_eps >= 0.0))
    return fail(GES_ERR_INVALID_ARG, "Adam or model constants out of range");
  if (runs == 0) return GES_OK;
  ges_status st = use_device(ctx->device);
  if (st != GES_OK) return st;
  FitArgs A;
  std::memset(&A, 0, sizeof(A));
  A.n = p->n_components;
  A.rows = p->model == GES_MIX_GEF ? 4 : 3;
  A.positive = p->positive_weights ? 1 : 0;
  A.epochs = p->epochs;
  A.n_points = n_points;
  A.y_stride = y_stride;
  A.lr = p->lr;
  A.b1 = p->beta1;
  A.b2 = p->beta2;
  A.adam_eps = p->adam_eps;
  A.nu = p->nu;
  A.mix_eps = p->mix_eps;
  A.x = x;
  A.y = y;
  A.params = params;
  A.final_loss = final_loss;
  A.grad = grad;
  A.loss_hist = loss_hist;
  cudaStream_t s = (cudaStream_t)stream;
  cudaError_t e;
  {
    TraceScope tr(ctx, "k_fit1d", s);
    e = p->precision == 32 ? launch_fit_model<float>(p->model, A, runs, s) : launch_fit_model<double>(p->model, A, runs, s);
  }
  count_launches(1);
  return e == cudaSuccess ? GES_OK : cuda_fail(e, "fit1d launch");
}

}  // extern "C"
