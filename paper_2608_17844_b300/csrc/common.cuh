// Shared device helpers: complex arithmetic on float2/double2, the
// precision traits that let one kernel body serve the FP32 (c64) and FP64
// (c128) paths, and small PTX wrappers (mbarrier, bulk copy, timers).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MOMA_DEV __device__ __forceinline__
#define MOMA_HD __host__ __device__ __forceinline__

// ---- double-FP32 ("dfl") arithmetic -------------------------------------
// A value hi + lo of two floats with |lo| <= ulp(hi) / 2: about 48
// significant bits (relative rounding ~2^-47), carried on the FP32 pipes.
// B300 runs FP64 at ~1/58 of its FP32 rate, so the FP64-bound stages of
// the mixed path (block-bin transform, residual bin product and FFTs)
// compute in dfl.  Built from error-free transformations: Knuth's
// two-sum, Dekker's fast two-sum (|a| >= |b|) and the FMA two-product;
// every step uses the _rn intrinsics so that the compiler cannot contract
// or reassociate them.  Addition is the "sloppy" variant (one two-sum on
// the high parts), whose error is bounded by ~2^-46 (|a| + |b|): enough for
// sums of products and FFT butterflies, whose error analysis is normwise.
struct dfl {
  float hi, lo;
  dfl() = default;
  MOMA_HD constexpr dfl(float h, float l) : hi(h), lo(l) {}
  MOMA_HD constexpr dfl(float v) : hi(v), lo(0.0f) {}
  MOMA_HD dfl(double v) : hi((float)v), lo((float)(v - (double)(float)v)) {}
  MOMA_HD dfl(int v) : dfl((double)v) {}
  MOMA_HD explicit operator double() const { return (double)hi + (double)lo; }
};
struct __align__(16) dfl2 {
  dfl x, y;
};

#ifdef __CUDACC__
MOMA_DEV dfl df_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bp = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bp)), __fsub_rn(b, bp));
  return dfl(s, e);
}
MOMA_DEV dfl df_fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfl(s, __fsub_rn(b, __fsub_rn(s, a)));
}
MOMA_DEV dfl operator+(dfl a, dfl b) {
  const dfl s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}
MOMA_DEV dfl operator-(dfl a) { return dfl(-a.hi, -a.lo); }
MOMA_DEV dfl operator-(dfl a, dfl b) { return a + (-b); }
MOMA_DEV dfl operator*(dfl a, dfl b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  return df_fast_two_sum(p, e);
}
// c + a*b with one renormalisation.
MOMA_DEV dfl fma(dfl a, dfl b, dfl c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const dfl s = df_two_sum(c.hi, p);
  return df_fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}
MOMA_DEV dfl operator/(dfl a, dfl b) {
  const float q1 = __fdiv_rn(a.hi, b.hi);
  const dfl r = a - b * dfl(q1, 0.0f);
  return df_fast_two_sum(q1, __fdiv_rn(r.hi, b.hi));
}
// Square root: one Newton correction of the float root, s + (a - s^2) / 2s.
MOMA_DEV dfl dsqrt(dfl a) {
  const float s = sqrtf(a.hi);
  if (!(s > 0.0f)) return dfl(s, 0.0f);
  const float p = __fmul_rn(s, s);
  const float e = __fmaf_rn(s, s, -p);  // s*s = p + e exactly
  const float r = __fadd_rn(__fsub_rn(__fsub_rn(a.hi, p), e), a.lo);
  return df_fast_two_sum(s, __fdiv_rn(r, __fmul_rn(2.0f, s)));
}
MOMA_DEV dfl &operator+=(dfl &a, dfl b) { return a = a + b; }
// Unnormalised double-FP32 accumulator (value s + t) for sums of products:
// each product's high part joins s through an exact two-sum, the rounding
// error of that sum and the product's error (FMA two-product) gather in t,
// and one two-sum at the end renormalises.  Against a renormalised `fma`
// per term this saves a fast two-sum per term; every step that was exact
// stays exact.
struct DfAcc {
  float s, t;
};
MOMA_DEV DfAcc dfacc(dfl c) { return DfAcc{c.hi, c.lo}; }
MOMA_DEV void dfacc_fma(DfAcc &acc, dfl a, dfl b) {  // acc += a b
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
  const dfl q = df_two_sum(acc.s, p);
  acc.s = q.hi;
  acc.t = __fadd_rn(acc.t, __fadd_rn(q.lo, e));
}
MOMA_DEV void dfacc_add(DfAcc &acc, DfAcc b) {  // acc += b
  const dfl q = df_two_sum(acc.s, b.s);
  acc.s = q.hi;
  acc.t = __fadd_rn(acc.t, __fadd_rn(q.lo, b.t));
}
MOMA_DEV dfl dfacc_value(DfAcc acc) { return df_two_sum(acc.s, acc.t); }

MOMA_DEV dfl &operator*=(dfl &a, dfl b) { return a = a * b; }
#endif

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };
template <> struct Cplx<dfl> { using T = dfl2; };

MOMA_HD float2 mk(float a, float b) { return make_float2(a, b); }
MOMA_HD double2 mk(double a, double b) { return make_double2(a, b); }
MOMA_HD dfl2 mk(dfl a, dfl b) { dfl2 r; r.x = a; r.y = b; return r; }

template <typename C> MOMA_HD C cadd(C a, C b) { C r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <typename C> MOMA_HD C csub(C a, C b) { C r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <typename C> MOMA_HD C cmul(C a, C b) {
  C r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// acc + a*b
template <typename C> MOMA_HD C cfma(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(a.y, b.x, acc.y);
  return acc;
}
// acc + conj(a)*b
template <typename C> MOMA_HD C cfmac(C a, C b, C acc) {
  acc.x = fma(a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
// acc - a*conj(b), four fused multiply-adds
template <typename C> MOMA_HD C cfms_conj(C a, C b, C acc) {
  acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(-a.y, b.x, acc.y); acc.y = fma(a.x, b.y, acc.y);
  return acc;
}
// acc - a*b, four fused multiply-adds
template <typename C> MOMA_HD C cfms(C a, C b, C acc) {
  acc.x = fma(-a.x, b.x, acc.x); acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(-a.x, b.y, acc.y); acc.y = fma(-a.y, b.x, acc.y);
  return acc;
}
template <typename C> MOMA_HD C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename S> MOMA_HD C cscale(C a, S s) { a.x *= s; a.y *= s; return a; }
// multiply by -i and +i
template <typename C> MOMA_HD C cmul_mi(C a) { C r; r.x = a.y; r.y = -a.x; return r; }
template <typename C> MOMA_HD C cmul_pi(C a) { C r; r.x = -a.y; r.y = a.x; return r; }

template <typename C> MOMA_HD C czero() { C r; r.x = 0; r.y = 0; return r; }

// Conversions between the storage precisions.
MOMA_HD float2 to_c(float2 v, float2*) { return v; }
MOMA_HD float2 to_c(double2 v, float2*) { return make_float2((float)v.x, (float)v.y); }
MOMA_HD double2 to_c(float2 v, double2*) { return make_double2(v.x, v.y); }
MOMA_HD double2 to_c(double2 v, double2*) { return v; }
MOMA_HD dfl2 to_c(float2 v, dfl2*) { dfl2 r; r.x = dfl(v.x); r.y = dfl(v.y); return r; }
MOMA_HD dfl2 to_c(double2 v, dfl2*) { dfl2 r; r.x = dfl(v.x); r.y = dfl(v.y); return r; }
MOMA_HD dfl2 to_c(dfl2 v, dfl2*) { return v; }
MOMA_HD float2 to_c(dfl2 v, float2*) { return make_float2(v.x.hi + v.x.lo, v.y.hi + v.y.lo); }
MOMA_HD double2 to_c(dfl2 v, double2*) { return make_double2((double)v.x, (double)v.y); }
template <typename Cout, typename Cin> MOMA_HD Cout cvt(Cin v) { return to_c(v, (Cout*)nullptr); }

MOMA_DEV float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
MOMA_DEV double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
MOMA_DEV dfl shfl_xor(dfl v, int m) {
  return dfl(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

template <typename C> MOMA_DEV C warp_sum(C v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) { v.x += shfl_xor(v.x, m); v.y += shfl_xor(v.y, m); }
  return v;
}
MOMA_DEV double warp_sum(double v) {
#pragma unroll
  for (int m = 16; m > 0; m >>= 1) v += shfl_xor(v, m);
  return v;
}

MOMA_DEV uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// ---- mbarrier / bulk-copy wrappers (sm_90+ PTX, used on sm_103a) --------
MOMA_DEV uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

MOMA_DEV void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
MOMA_DEV void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
MOMA_DEV void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

MOMA_DEV void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
MOMA_DEV bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait: gives up after `limit_ns` nanoseconds and returns false.
MOMA_DEV bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  uint64_t t0 = global_ns();
  for (uint32_t it = 0;; ++it) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && global_ns() - t0 > limit_ns) return false;
  }
}
// One-dimensional bulk copy global -> shared, completion counted on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
MOMA_DEV void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Device-side error bits reported back to the host.
enum : unsigned {
  DEVERR_TIMEOUT = 1u,
  DEVERR_NOT_PD = 2u,
  DEVERR_NONFINITE = 4u,
};
