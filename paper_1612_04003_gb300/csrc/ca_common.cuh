// ca_common.cuh -- device helpers shared by the CA-BCD / CA-BDCD kernels (sm_103a).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

// Device error word bits (read back by the host after a solve).
#define CA_DEV_ERR_NOT_SPD 1u
#define CA_DEV_ERR_NONFINITE 2u
#define CA_DEV_ERR_TIMEOUT 4u
#define CA_DEV_ERR_ARG 8u

// Bounded waits give up after this much wall time (ns, %globaltimer).
#define CA_WAIT_LIMIT_NS 2000000000ull

__device__ __forceinline__ void ca_flag(unsigned* err, unsigned bit) { atomicOr(err, bit); }

__device__ __forceinline__ uint64_t ca_globaltimer() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---------------------------------------------------------------------------
// Sampling rule: Philox4x64-10 (Salmon, Moraes, Dror, Shaw, SC'11) feeding
// Floyd's subset algorithm.  Ten rounds; round r uses the key bumped r times
// by the Weyl increments.
// ---------------------------------------------------------------------------
struct Philox4x64Key {
  uint64_t k0, k1;
};

__device__ __forceinline__ void ca_philox4x64_10(uint64_t (&x)[4], Philox4x64Key key) {
  const uint64_t mA = 0xD2E7470EE14C6C93ull, mB = 0xCA5A826395121157ull;
  const uint64_t wA = 0x9E3779B97F4A7C15ull, wB = 0xBB67AE8584CAA73Bull;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint64_t pa_lo = mA * x[0], pa_hi = __umul64hi(mA, x[0]);
    const uint64_t pb_lo = mB * x[2], pb_hi = __umul64hi(mB, x[2]);
    const uint64_t y0 = pb_hi ^ x[1] ^ key.k0;
    const uint64_t y2 = pa_hi ^ x[3] ^ key.k1;
    x[0] = y0;
    x[1] = pb_lo;
    x[2] = y2;
    x[3] = pa_lo;
    key.k0 += wA;
    key.k1 += wB;
  }
}

// ---------------------------------------------------------------------------
// mbarrier / cp.async / proxy fences (PTX ISA 8.x)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile(
      "{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the barrier phase with the given parity; gives up after limit_ns,
// flags CA_DEV_ERR_TIMEOUT and returns false.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, unsigned* err,
                                                  uint64_t limit_ns = CA_WAIT_LIMIT_NS) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = ca_globaltimer();
  for (uint32_t it = 1;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 0u && ca_globaltimer() - t0 > limit_ns) {
      ca_flag(err, CA_DEV_ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void cp_async_16_zfill(uint32_t dst, const void* src, uint32_t src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(src_bytes)
               : "memory");
}

__device__ __forceinline__ void cp_async_8(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_4(uint32_t dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(dst), "l"(src) : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// 1/d by Newton-Raphson, r <- r (2 - d r), from the FP32 reciprocal: each step
// doubles the correct bits (about 23 -> 46 -> full FP64).  d must be a
// normal FP32-representable magnitude; otherwise the FP64 division is used.
__device__ __forceinline__ double rcp_newton(double d) {
  const float f = (float)d;
  double r = (double)__frcp_rn(f);
  if (!(fabs(r) > 0.0) || !isfinite(r)) return 1.0 / d;
  r = r * fma(-d, r, 2.0);
  r = r * fma(-d, r, 2.0);
  return r;
}

// Programmatic dependent launch: wait until the preceding grid in the stream
// has completed (its memory visible); no-op without a programmatic dependency.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
// Let the next grid in the stream (if launched as a programmatic dependent)
// start scheduling its CTAs.
__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// ---------------------------------------------------------------------------
// Packed lower-triangle index: e -> (i, j) with j <= i, e = i(i+1)/2 + j.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void tri_decode(long long e, int& i, int& j) {
  // single-precision estimate (FP64 is scarce on this part), integer fix-up
  long long r = (long long)((sqrtf(8.0f * (float)e + 1.0f) - 1.0f) * 0.5f);
  while (r * (r + 1) / 2 > e) --r;
  while ((r + 1) * (r + 2) / 2 <= e) ++r;
  i = (int)r;
  j = (int)(e - r * (r + 1) / 2);
}

// Knuth's TwoSum: s + e == a + b exactly (round-to-nearest FP32, no
// reassociation).  Used for compensated FP32 sums where FP64 would be slow.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// hi + lo += x (compensated accumulation)
__device__ __forceinline__ void comp_add(float& hi, float& lo, float x) {
  float s, e;
  two_sum(hi, x, s, e);
  hi = s;
  lo += e;
}

// x = hi + lo with hi = fp32(x), lo = fp32(x - hi)
__device__ __forceinline__ float2 split_f64(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}

// Double-float arithmetic: a value is hi + lo (two FP32, |lo| <= ulp(hi)/2);
// Dekker / Knuth error-free transformations give ~2^-44 relative accuracy
// on the FP32 pipe, which on this part is ~64x faster than the FP64 pipe.
__device__ __forceinline__ float2 df_add(float2 a, float2 b) {
  float s, e;
  two_sum(a.x, b.x, s, e);
  e += a.y + b.y;
  const float h = s + e;
  return make_float2(h, e - (h - s));
}

__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// (hi, lo) from a compensated-sum pair whose lo may exceed ulp(hi)/2
__device__ __forceinline__ float2 df_norm(float hi, float lo) {
  const float h = hi + lo;
  return make_float2(h, lo - (h - hi));
}

__device__ __forceinline__ float2 df_mul(float2 a, float2 b) {
  const float p = a.x * b.x;
  const float e = fmaf(a.x, b.x, -p) + fmaf(a.x, b.y, a.y * b.x);
  const float h = p + e;
  return make_float2(h, e - (h - p));
}

// 1/d for a positive double-float d: the hardware reciprocal estimate r
// (rcp.approx, within 1 ulp) refined by one Newton step r + r e with the
// residual e = 1 - d r formed by a fused multiply-add (|e| <= 2^-22, so the
// FMA's single rounding leaves it accurate to ~2^-46 of 1) and the low part of
// d; the result (r, r e) is a normalised double-float, ~2^-44 relative.
__device__ __forceinline__ float2 df_rcp(float2 d) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d.x));
  const float e = fmaf(-d.y, r, fmaf(-d.x, r, 1.0f));
  const float lo = r * e;
  const float h = r + lo;
  return make_float2(h, lo - (h - r));
}

// (hi, lo) += x * (dh + dl) for an FP32 x and a double-float (dh, dl): the
// product x dh is split exactly into p + e (e by a fused multiply-add), p is
// accumulated by TwoSum and the small terms e and x dl go to lo (the
// compensated dot product of Ogita, Rump and Oishi, 2005).  The sum carries
// ~2^-44 of sum |x (dh + dl)|, against 2^-24 when products are rounded.
__device__ __forceinline__ void df_dot_acc(float x, float dh, float dl, float& hi, float& lo) {
  const float p = x * dh;
  const float e = fmaf(x, dl, fmaf(x, dh, -p));
  float s, t;
  two_sum(hi, p, s, t);
  hi = s;
  lo += t + e;
}

__device__ __forceinline__ float2 df_shfl_xor(float2 v, int o) {
  return make_float2(__shfl_xor_sync(0xffffffffu, v.x, o), __shfl_xor_sync(0xffffffffu, v.y, o));
}

// (shi, slo) += a * b, with a and b double-float values
__device__ __forceinline__ void df_fma_acc(float2 a, float2 b, float& shi, float& slo) {
  const float p = a.x * b.x;
  const float e = fmaf(a.x, b.x, -p);                 // exact low part of a.x*b.x
  const float cross = fmaf(a.x, b.y, a.y * b.x);      // first-order terms
  float s, t;
  two_sum(shi, p, s, t);
  shi = s;
  slo += t + (e + cross);
}

// Solve constants of one outer step in the common form
//   (cG R_jj + cI I) Delta_j = cP p_j - cI x[I_j] - cY yv[I_j] - cG sum_{t<j} R_jt Delta_t
// primal (Alg. 2): cG = 1/n, cI = lambda, cP = 1/n, cY = 0, x = w
// dual   (Alg. 4): cG = 1/(lambda n), cI = 1, cP = 1, cY = 1, x = alpha, yv = y
struct SolveArgs {
  const int* idx;   // s' * b sampled indices (row order of Y)
  long long N;      // length of x (indices are checked against it)
  int b, s_cur, sb, ldr;  // block size, blocks this outer step, s'*b, leading dim of R
  double cG, cI, cP, cY;
  double* x;        // w (primal) or alpha (dual), updated in place at I_j
  const double* yv; // y (dual) or nullptr
  double* delta;    // out: Delta (s'*b)
};
