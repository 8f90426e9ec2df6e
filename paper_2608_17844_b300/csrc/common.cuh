// Shared device helpers: complex arithmetic on float2/double2, the
// precision traits that let one kernel body serve the FP32 (c64) and FP64
// (c128) paths, and small PTX wrappers (mbarrier, bulk copy, timers).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define MOMA_DEV __device__ __forceinline__
#define MOMA_HD __host__ __device__ __forceinline__

template <typename R> struct Cplx;
template <> struct Cplx<float> { using T = float2; };
template <> struct Cplx<double> { using T = double2; };

MOMA_HD float2 mk(float a, float b) { return make_float2(a, b); }
MOMA_HD double2 mk(double a, double b) { return make_double2(a, b); }

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
template <typename Cout, typename Cin> MOMA_HD Cout cvt(Cin v) { return to_c(v, (Cout*)nullptr); }

MOMA_DEV float shfl_xor(float v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }
MOMA_DEV double shfl_xor(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

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
