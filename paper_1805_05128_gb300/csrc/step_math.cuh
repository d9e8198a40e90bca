// step_math.cuh -- per-particle arithmetic shared by the step kernels and
// the pair-list kernel's fused second kick: order keys of doubles, the size
// d = (m / rho)^(1/D), the half-kick update, the FP32 sound speed and the CFL
// key of a particle.
#pragma once

#include <cstring>

#include "csph_internal.cuh"

namespace csph {

// Reductions run on order-preserving 64-bit integer keys of the doubles
// (integer ALU instead of the narrow FP64 pipe): key(x) = bits(x) for x >= 0,
// bits(x) ^ 0x7fff...f for x < 0, so key order is numeric order.
__device__ __forceinline__ long long dkey(double x) {
  long long b = __double_as_longlong(x);
  return b < 0 ? b ^ 0x7fffffffffffffffLL : b;
}
__device__ __forceinline__ double dunkey(long long k) {
  return __longlong_as_double(k < 0 ? k ^ 0x7fffffffffffffffLL : k);
}

// Conversions between FP64 and FP32 on the integer ALU.  The F2F
// conversions run on the narrow FP64 pipe, about as many of them as FP64
// additions and multiplies in the per-particle kernels of a mixed step.
// f32_rn(x) is x rounded to the nearest FP32 value, ties to even (IEEE 754
// roundTiesToEven), built from x's bits: the exponent rebiased from 1023 to
// 127, the 52-bit fraction cut to 23 bits and rounded on the 29 bits dropped;
// a carry out of the fraction moves into the exponent (up to infinity, which
// is the rounded value there).  Zeros keep their sign; other values outside
// FP32's normal range (subnormal results, infinities, NaN) take the F2F
// conversion.
__host__ __device__ __forceinline__ float f32_rn(double x) {
#ifdef __CUDA_ARCH__
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
#else
  unsigned long long bb;
  memcpy(&bb, &x, 8);
  const unsigned hi = (unsigned)(bb >> 32), lo = (unsigned)bb;
#endif
  const unsigned h = hi & 0x7fffffffu;
  unsigned r;
  if (h - (897u << 20) < ((1151u - 897u) << 20)) {         // 2^-126 <= |x| < 2^128
    r = ((h - (896u << 20)) << 3) | (lo >> 29);
    const unsigned rem = lo & 0x1fffffffu;
    r += (rem > 0x10000000u || (rem == 0x10000000u && (r & 1u))) ? 1u : 0u;
  } else if ((h | lo) == 0u) {
    r = 0u;
  } else {
    return (float)x;
  }
  r |= hi & 0x80000000u;
#ifdef __CUDA_ARCH__
  return __uint_as_float(r);
#else
  float f;
  memcpy(&f, &r, 4);
  return f;
#endif
}

// f64_of(f) is f as an FP64 value (exact): the exponent rebiased, the
// fraction moved up by 29 bits; zeros keep their sign, subnormals,
// infinities and NaN take the F2F conversion.
__host__ __device__ __forceinline__ double f64_of(float f) {
#ifdef __CUDA_ARCH__
  const unsigned u = __float_as_uint(f);
#else
  unsigned u;
  memcpy(&u, &f, 4);
#endif
  const unsigned a = u & 0x7fffffffu;
  unsigned hi, lo;
  if (a - 0x00800000u < 0x7f800000u - 0x00800000u) {
    hi = ((a >> 3) + (896u << 20)) | (u & 0x80000000u);
    lo = a << 29;
  } else if (a == 0u) {
    hi = u;
    lo = 0u;
  } else {
    return (double)f;
  }
#ifdef __CUDA_ARCH__
  return __hiloint2double((int)hi, (int)lo);
#else
  const unsigned long long bb = ((unsigned long long)hi << 32) | lo;
  double d;
  memcpy(&d, &bb, 8);
  return d;
#endif
}

// Reference velocity of a mixed pack: t = trunc(v) with |t| <= 32767, built
// from v's bits by integer operations (no FP64 arithmetic), and k = t as an
// int.  v - t is then exact in FP64 (|v - t| < 1 unless clamped) and rounds
// to FP32 with an error ~6e-8 of itself.  NaN and infinity clamp like large
// values, and their difference stays non-finite.
__device__ __forceinline__ double trunc_ref(double v, int& k) {
  const long long b = __double_as_longlong(v);
  const int e = (int)((b >> 52) & 0x7ff) - 1023;       // unbiased exponent
  if (e < 0) {                                          // |v| < 1
    k = 0;
    return 0.0;
  }
  if (e >= 15) {                                        // |v| >= 32768
    k = b < 0 ? -32767 : 32767;
    return b < 0 ? -32767.0 : 32767.0;
  }
  const int fb = 52 - e;                                // fraction bits below the binary point
  const int m = (int)(((b & 0xfffffffffffffLL) | (1LL << 52)) >> fb);
  k = b < 0 ? -m : m;
  return __longlong_as_double(b & ~((1LL << fb) - 1));
}

// Cube root in FP64 with little FP64 work: the FP32 cube root as seed, then
// two Newton steps on y^3 - x = 0 whose derivative reciprocal 1/(3 y^2) is
// taken in FP32 (a ~1e-7 relative error in the slope only scales each
// correction, so the error falls ~1e-7-fold per step to rounding level).
__device__ __forceinline__ double cbrt_fast(double x) {
  if (!(x > 1e-30 && x < 1e30)) return cbrt(x);   // outside the FP32 seed's comfortable range
  double y = (double)cbrtf((float)x);
  const double r = (double)__frcp_rn((float)(3.0 * y * y));
  y = y - (y * y * y - x) * r;
  y = y - (y * y * y - x) * r;
  return y;
}

__device__ __forceinline__ double size_of(int dim, double m, double rho) {
  double vol = m / rho;
  return dim == 1 ? vol : (dim == 2 ? sqrt(vol) : cbrt_fast(vol));
}

// d = (m / rho)^(1/D) for a mixed-precision step, in FP32 (relative error
// ~2e-7) from the FP64 mass and density: the step's pair decisions take this
// d as given (the FP32 packs and the FP64 exact test read the same stored
// value) and its FP32 fluxes are far coarser, while FP64 divisions, roots and
// conversions are what bound the per-particle kernels on GB300.  Volumes
// outside FP32's normal range take the FP64 path.
__device__ __forceinline__ double size_of_mixed(int dim, double m, double rho) {
  const float vf = __fdiv_rn(f32_rn(m), f32_rn(rho));
  if (!(vf > 1e-36f && vf < 1e36f)) return size_of(dim, m, rho);
  return f64_of(dim == 1 ? vf : (dim == 2 ? sqrtf(vf) : cbrtf(vf)));
}

// Half kick / drift y + a x: the oracle's correctly rounded product and sum
// for an FP64 handle; one fused multiply-add for a mixed handle (FP64 is the
// narrow pipe on this GPU and these kernels are bound by it).
template <bool MIXED>
__device__ __forceinline__ double axpy(double a, double x, double y) {
  if constexpr (MIXED) return __fma_rn(a, x, y);
  else return __dadd_rn(y, __dmul_rn(a, x));
}

// isfinite on the bits (integer ALU, not the FP64 pipe)
__device__ __forceinline__ bool finite_bits(double x) {
  return (__double_as_longlong(x) & 0x7ff0000000000000LL) != 0x7ff0000000000000LL;
}

// Sound speed in FP32 from an FP64 specific internal energy (the closures of
// eos() written in single precision; the stiffened gas in the form
// c^2 = gamma (gamma - 1)(rho e - P_inf) / rho, without the P + P_inf
// cancellation).  For the CFL bound of a mixed-precision step only.
__device__ __forceinline__ float sound_speed_f32(const Mat& m, float rho, float e) {
  const float g = m.gamma_f;
  float c2;
  if (m.eos == SPH_EOS_IDEAL) {
    c2 = g * (g - 1.0f) * e;
  } else if (m.eos == SPH_EOS_STIFFENED) {
    c2 = g * (g - 1.0f) * (rho * e - m.p_inf_f) / rho;
  } else if (m.eos == SPH_EOS_TAIT) {
    const float c0 = m.c0_f, r = rho / m.rho0_f;
    c2 = c0 * c0 * (m.tait_n > 1 ? ipow(r, m.tait_n - 1) : (m.tait_n == 1 ? 1.0f : powf(r, g - 1.0f)));
  } else {
    const float ca = m.c0_f, sa = m.s_a_f, r0 = m.rho0_f;
    const float x = r0 / rho, u = 1.0f - x, D = 1.0f - sa * u, iD2 = 1.0f / (D * D);
    const float Pr = r0 * ca * ca * u * iD2, er = 0.5f * ca * ca * u * u * iD2;
    const float du = x / rho;
    const float dPr = r0 * ca * ca * (1.0f + sa * u) * iD2 / D * du;
    const float der = ca * ca * u * iD2 / D * du;
    const float P = Pr + g * rho * (e - er);
    c2 = dPr + g * (e - er) - g * rho * der + g * P / rho;
  }
  return c2 > 0.0f ? sqrtf(c2) : 0.0f;
}

// ---------------------------------------------------------------------------
// The CFL bound dt_i = eta d_i / (c_i + |v_i|).  Inside a mixed-precision step
// (no bbox, nothing written back) it is evaluated in FP32 from the FP64 state
// (e = E - v^2/2 in FP64): it is a stability bound, the step then uses that dt
// exactly in FP64, and the FP64 divisions, roots and cube root of every
// particle are what bound these kernels on GB300.  FP64 handles keep the FP64
// expression (bit parity of dt).
// ---------------------------------------------------------------------------
// CFL order key of one particle's bound dt_i = eta d_i / (c_i + |v_i|) at the
// given state: FP32 in a mixed-precision handle (see above), FP64 otherwise.
__device__ __forceinline__ long long cfl_key(const DevParams& P, double vx, double vy, double vz, double E,
                                             double rho, double m, int mi) {
  const double v2 = vx * vx + vy * vy + vz * vz;
  const double e = E - 0.5 * v2;
  if (P.precision == SPH_PREC_MIXED) {
    const float rf = (float)rho;
    const float c = sound_speed_f32(P.mat[mi], rf, (float)e);
    const float vol = (float)m / rf;
    const float d = P.dim == 1 ? vol : (P.dim == 2 ? sqrtf(vol) : cbrtf(vol));
    return dkey((double)(P.eta_f * d / (c + sqrtf((float)v2))));
  }
  double Pp, cp;
  eos(P.mat[mi], rho, e, Pp, cp);
  return dkey((P.eta * size_of(P.dim, m, rho)) / (cp + sqrt(v2)));
}

}  // namespace csph
