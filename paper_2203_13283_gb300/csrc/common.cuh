// Shared device/host helpers of the Woodbury-circulant solver library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>

#define WCS_PI 3.14159265358979323846
#define WCS_EULER_GAMMA 0.57721566490153286061

// ---------------------------------------------------------------------------
// Minimal complex arithmetic (double and float), interleaved (re, im) layout.
// ---------------------------------------------------------------------------
struct __align__(16) zd {
  double x, y;
};
struct __align__(8) zf {
  float x, y;
};

// Coefficients of the fixed-length Hankel expansion for x >= 20 (see
// hankel01_asymptotic_fixed): (-1)^m a_k(nu) for the real argument and
// (-1)^m a_k(nu) (1 + i t)^-k for x (1 + i t), k = 2m (re, ce) and 2m + 1 (ro, co).
constexpr int ASYM_M = 10;
struct AsymCoef {
  double re[2][ASYM_M], ro[2][ASYM_M];
  zd ce[2][ASYM_M], co[2][ASYM_M];
};

// k~ = k (1 + i t): per-run constants for evaluating both wavenumbers of a
// point pair from one real argument x = k R.  Passed to the kernels by value
// (not as __constant__ data), so contexts on different streams can assemble
// different contours at the same time.
struct KtPair {
  double t = 0.0;
  zd c1;   // 1 / (1 + i t)
  zd c2;   // (1 + i t)^(-1/2), principal branch
  AsymCoef asym;
  // x above which 4, 6, 8, 10, 14 terms of the expansion meet the run's
  // tolerance (below xth[4]: all 2 ASYM_M terms); see set_asym_terms
  double xth[5] = {1e300, 1e300, 1e300, 1e300, 1e300};
};


__host__ __device__ __forceinline__ zd mkz(double a, double b = 0.0) { zd r; r.x = a; r.y = b; return r; }
__host__ __device__ __forceinline__ zd operator+(zd a, zd b) { return mkz(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ zd operator-(zd a, zd b) { return mkz(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ zd operator-(zd a) { return mkz(-a.x, -a.y); }
__host__ __device__ __forceinline__ zd operator*(zd a, zd b) {
  return mkz(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__host__ __device__ __forceinline__ zd operator*(double s, zd a) { return mkz(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ zd operator*(zd a, double s) { return mkz(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ zd& operator+=(zd& a, zd b) { a.x += b.x; a.y += b.y; return a; }
__host__ __device__ __forceinline__ zd& operator-=(zd& a, zd b) { a.x -= b.x; a.y -= b.y; return a; }
__host__ __device__ __forceinline__ zd conj(zd a) { return mkz(a.x, -a.y); }
__host__ __device__ __forceinline__ double abs2(zd a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ double zabs(zd a) { return hypot(a.x, a.y); }
__host__ __device__ __forceinline__ zd zdiv(zd a, zd b) {
  // Smith's algorithm
  if (fabs(b.x) >= fabs(b.y)) {
    double r = b.y / b.x, d = b.x + r * b.y;
    return mkz((a.x + r * a.y) / d, (a.y - r * a.x) / d);
  }
  double r = b.x / b.y, d = b.y + r * b.x;
  return mkz((a.x * r + a.y) / d, (a.y * r - a.x) / d);
}
__host__ __device__ __forceinline__ zd zrecip(zd b) { return zdiv(mkz(1.0, 0.0), b); }
__host__ __device__ __forceinline__ zd zlog(zd a) { return mkz(log(zabs(a)), atan2(a.y, a.x)); }
__host__ __device__ __forceinline__ zd zsqrt(zd a) {
  double r = zabs(a);
  if (r == 0.0) return mkz(0.0, 0.0);
  double t = sqrt(0.5 * (r + fabs(a.x)));
  if (a.x >= 0.0) return mkz(t, a.y / (2.0 * t));
  return mkz(fabs(a.y) / (2.0 * t), a.y >= 0.0 ? t : -t);
}
// fused complex multiply-add: acc += a * b
__host__ __device__ __forceinline__ void zfma(zd& acc, zd a, zd b) {
  acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
  acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc += s * b (s real)
__host__ __device__ __forceinline__ void zfmas(zd& acc, double s, zd b) {
  acc.x = fma(s, b.x, acc.x);
  acc.y = fma(s, b.y, acc.y);
}

// ---------------------------------------------------------------------------
// Error plumbing shared by the host-side translation units.
// ---------------------------------------------------------------------------
#ifndef __CUDACC_RTC__
#include <atomic>
#include <string>
namespace wcs {
void set_error(const std::string& msg);
// host-side count of kernel launches issued by the library (any thread)
extern std::atomic<unsigned long long> g_launches;
inline void note_launch() { ++g_launches; }
}
#define WCS_CUDA_TRY(expr)                                                        \
  do {                                                                            \
    cudaError_t _e = (expr);                                                      \
    if (_e != cudaSuccess) {                                                      \
      wcs::set_error(std::string(#expr) + ": " + cudaGetErrorString(_e));         \
      return WCS_ERR_CUDA;                                                        \
    }                                                                             \
  } while (0)
#define WCS_LAUNCH_CHECK()                                                        \
  do {                                                                            \
    cudaError_t _e = cudaGetLastError();                                          \
    if (_e != cudaSuccess) {                                                      \
      wcs::set_error(std::string("kernel launch: ") + cudaGetErrorString(_e));    \
      return WCS_ERR_CUDA;                                                        \
    }                                                                             \
  } while (0)
#endif
