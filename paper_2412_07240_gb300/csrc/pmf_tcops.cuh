// Building blocks of the tcgen05 kernels (included by the 2-D and 3-D
// tensor-core translation units): PTX wrappers, the no-swizzle canonical
// operand layout, split-precision operand stores.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pmf_internal.cuh"

namespace pmf {
namespace {

constexpr int kPlane = 32768;                // bytes of one 16-bit operand plane
constexpr long long kSpin = 1LL << 22;       // bounded mbarrier polls

// --- PTX wrappers ------------------------------------------------------------
__device__ __forceinline__ uint32_t su32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// kind::f16 / kind::tf32 instruction descriptor, FP32 accumulate, M = 128.
__device__ __forceinline__ uint32_t idesc(int fmt, int a_mn, int n) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)a_mn << 15) |
         ((uint32_t)(n >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}" ::"r"(d),
               "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
               "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar));
}

__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t phase, long long polls = kSpin) {
  uint32_t done = 0;
  for (long long it = 0; it < polls; ++it) {
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}"
                 : "=r"(done) : "r"(mbar), "r"(phase));
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar) : "memory");
}

__device__ __forceinline__ void expect_tx(uint32_t mbar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
}

// Four consecutive accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ float4 tmem_ld4(uint32_t taddr) {
  uint32_t r0, r1, r2, r3;
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];\n"
               "tcgen05.wait::ld.sync.aligned;"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(taddr)
               : "memory");
  return make_float4(__uint_as_float(r0), __uint_as_float(r1), __uint_as_float(r2), __uint_as_float(r3));
}

// Columns [0, ncol) (ncol a multiple of 4, at most 32, the same in the whole
// warp) of this thread's TMEM lane from taddr into v[0..ncol/4); v[j] beyond
// are zero.  All loads are in flight together; the wait names the registers
// so that no use of them is scheduled before it.
__device__ __forceinline__ void tmem_ld_cols(uint32_t taddr, int ncol, float4 (&v)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    if (j * 4 < ncol) {
      uint32_t r0, r1, r2, r3;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                   : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                   : "r"(taddr + 4 * j)
                   : "memory");
      v[j] = make_float4(__uint_as_float(r0), __uint_as_float(r1), __uint_as_float(r2), __uint_as_float(r3));
    } else {
      v[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0].x), "+f"(v[0].y), "+f"(v[0].z), "+f"(v[0].w), "+f"(v[1].x), "+f"(v[1].y),
                 "+f"(v[1].z), "+f"(v[1].w), "+f"(v[2].x), "+f"(v[2].y), "+f"(v[2].z), "+f"(v[2].w),
                 "+f"(v[3].x), "+f"(v[3].y), "+f"(v[3].z), "+f"(v[3].w)::"memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[4].x), "+f"(v[4].y), "+f"(v[4].z), "+f"(v[4].w), "+f"(v[5].x), "+f"(v[5].y),
                 "+f"(v[5].z), "+f"(v[5].w), "+f"(v[6].x), "+f"(v[6].y), "+f"(v[6].z), "+f"(v[6].w),
                 "+f"(v[7].x), "+f"(v[7].y), "+f"(v[7].z), "+f"(v[7].w)::"memory");
}

// Columns [0, ncol) (ncol a multiple of 4, at most 16) of this thread's TMEM
// lane into v[0..ncol/4), zeros beyond; one wait for all loads.
__device__ __forceinline__ void tmem_ld_cols4(uint32_t taddr, int ncol, float4 (&v)[4]) {
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    if (j * 4 < ncol) {
      uint32_t r0, r1, r2, r3;
      asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                   : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                   : "r"(taddr + 4 * j)
                   : "memory");
      v[j] = make_float4(__uint_as_float(r0), __uint_as_float(r1), __uint_as_float(r2), __uint_as_float(r3));
    } else {
      v[j] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
  }
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+f"(v[0].x), "+f"(v[0].y), "+f"(v[0].z), "+f"(v[0].w), "+f"(v[1].x), "+f"(v[1].y),
                 "+f"(v[1].z), "+f"(v[1].w), "+f"(v[2].x), "+f"(v[2].y), "+f"(v[2].z), "+f"(v[2].w),
                 "+f"(v[3].x), "+f"(v[3].y), "+f"(v[3].z), "+f"(v[3].w)::"memory");
}

// Bulk copy shared -> global (bulk-group completion), commit, and wait for
// all of this thread's bulk groups to complete.
__device__ __forceinline__ void bulk_store(void* dst, uint32_t src, uint32_t bytes) {
  asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(src), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// ... until the shared-memory sources of this thread's bulk groups have been read
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Warm the L2 with [src, src + bytes) (16-byte aligned, multiple of 16 bytes).
__device__ __forceinline__ void prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// --- operand layout ------------------------------------------------------------
// Element (r, c) of a 128-row operand plane: 8-row x 16-byte core matrices,
// 16 (16-bit) or 32 (32-bit) core matrices per 8-row block.
template <int P>
struct Fmt;
template <>
struct Fmt<PMF_PREC_FP16X3> {
  static constexpr int esz = 2, rowblk = 2048, planes = 2, kper = 16, code = 0;
};
template <>
struct Fmt<PMF_PREC_BF16X3> {
  static constexpr int esz = 2, rowblk = 2048, planes = 2, kper = 16, code = 1;
};
template <>
struct Fmt<PMF_PREC_TF32> {
  static constexpr int esz = 4, rowblk = 4096, planes = 1, kper = 8, code = 2;
};
template <>
struct Fmt<PMF_PREC_BF16X6> {
  static constexpr int esz = 2, rowblk = 2048, planes = 3, kper = 16, code = 1;
};

// Operand tiles of a size class C (the largest axis they hold): an 8-row
// block covers C elements along K, so an R-row plane takes R * C * esz bytes
// (class 128, 16-bit: 32 KiB).  The MMA reads 128 rows (M) of the A operand;
// a kernel whose lanes >= R are never used keeps R < 128 rows per plane, and
// the rows the MMA reads past a plane fall into the next plane or region
// (garbage lanes, discarded).
template <int P, int C, int R = 128>
struct Lay {
  static constexpr int rowblk = C * Fmt<P>::esz * 8;
  static constexpr int plane = R * C * Fmt<P>::esz;     // an R-row (M) operand plane
  static constexpr int wplane = C * C * Fmt<P>::esz;    // a C-row matrix (W) plane
};

template <int P, int C = 128>
__device__ __forceinline__ uint32_t op_off(int r, int c) {
  constexpr int epc = 16 / Fmt<P>::esz;
  return (uint32_t)((r >> 3) * Lay<P, C>::rowblk + (c / epc) * 128 + (r & 7) * 16 + (c % epc) * Fmt<P>::esz);
}

__device__ __forceinline__ uint32_t h2u(__half2 h) { return *(uint32_t*)&h; }
__device__ __forceinline__ uint32_t b2u(__nv_bfloat162 h) { return *(uint32_t*)&h; }

// Elements (r, c..c+3) (c a multiple of 4) of the operand planes at base, scaled
// by s: split into hi + lo 16-bit planes, hi + mid + lo BF16 planes (BF16X6:
// x - hi and x - hi - mid are exact in float32, so the three pieces keep all
// 24 significand bits), or one float32 plane for TF32.
template <int P, int C = 128, bool kW = false, int R = 128>
__device__ __forceinline__ void store4(uint8_t* base, int r, int c, float4 v, float s) {
  constexpr int kPl = kW ? Lay<P, C>::wplane : Lay<P, C, R>::plane;
  v.x *= s;
  v.y *= s;
  v.z *= s;
  v.w *= s;
  const uint32_t off = op_off<P, C>(r, c);
  if constexpr (P == PMF_PREC_TF32) {
    *(float4*)(base + off) = v;
  } else if constexpr (P == PMF_PREC_FP16X3) {
    const __half2 h0 = __floats2half2_rn(v.x, v.y), h1 = __floats2half2_rn(v.z, v.w);
    const float2 f0 = __half22float2(h0), f1 = __half22float2(h1);
    const __half2 l0 = __floats2half2_rn(v.x - f0.x, v.y - f0.y), l1 = __floats2half2_rn(v.z - f1.x, v.w - f1.y);
    *(uint2*)(base + off) = make_uint2(h2u(h0), h2u(h1));
    *(uint2*)(base + kPl + off) = make_uint2(h2u(l0), h2u(l1));
  } else {
    const __nv_bfloat162 h0 = __floats2bfloat162_rn(v.x, v.y), h1 = __floats2bfloat162_rn(v.z, v.w);
    const float2 f0 = __bfloat1622float2(h0), f1 = __bfloat1622float2(h1);
    const float4 r = make_float4(v.x - f0.x, v.y - f0.y, v.z - f1.x, v.w - f1.y);
    const __nv_bfloat162 l0 = __floats2bfloat162_rn(r.x, r.y);
    const __nv_bfloat162 l1 = __floats2bfloat162_rn(r.z, r.w);
    *(uint2*)(base + off) = make_uint2(b2u(h0), b2u(h1));
    *(uint2*)(base + kPl + off) = make_uint2(b2u(l0), b2u(l1));
    if constexpr (P == PMF_PREC_BF16X6) {
      const float2 g0 = __bfloat1622float2(l0), g1 = __bfloat1622float2(l1);
      const __nv_bfloat162 e0 = __floats2bfloat162_rn(r.x - g0.x, r.y - g0.y);
      const __nv_bfloat162 e1 = __floats2bfloat162_rn(r.z - g1.x, r.w - g1.y);
      *(uint2*)(base + 2 * kPl + off) = make_uint2(b2u(e0), b2u(e1));
    }
  }
}

// Elements (r, c..c+7) (c a multiple of 8): one 16-byte store per plane for the
// 16-bit formats (a whole core-matrix row; the 8-byte stores of store4 leave
// half of each bank wavefront unused), two float32 stores for TF32.
template <int P, int C = 128, bool kW = false, int R = 128>
__device__ __forceinline__ void store8(uint8_t* base, int r, int c, float4 a, float4 b, float s) {
  if constexpr (P == PMF_PREC_TF32) {
    store4<P, C, kW, R>(base, r, c, a, s);
    store4<P, C, kW, R>(base, r, c + 4, b, s);
  } else {
    constexpr int kPl = kW ? Lay<P, C>::wplane : Lay<P, C, R>::plane;
    const float x[8] = {a.x * s, a.y * s, a.z * s, a.w * s, b.x * s, b.y * s, b.z * s, b.w * s};
    const uint32_t off = op_off<P, C>(r, c);
    uint32_t pc[3][4];
    if constexpr (P == PMF_PREC_FP16X3) {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const __half2 h = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
        const float2 f = __half22float2(h);
        pc[0][i] = h2u(h);
        pc[1][i] = h2u(__floats2half2_rn(x[2 * i] - f.x, x[2 * i + 1] - f.y));
      }
    } else {
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
        const float2 f = __bfloat1622float2(h);
        const float r0 = x[2 * i] - f.x, r1 = x[2 * i + 1] - f.y;
        const __nv_bfloat162 m = __floats2bfloat162_rn(r0, r1);
        pc[0][i] = b2u(h);
        pc[1][i] = b2u(m);
        if constexpr (P == PMF_PREC_BF16X6) {
          const float2 g = __bfloat1622float2(m);
          pc[2][i] = b2u(__floats2bfloat162_rn(r0 - g.x, r1 - g.y));
        }
      }
    }
#pragma unroll
    for (int pl = 0; pl < Fmt<P>::planes; ++pl)
      *(uint4*)(base + pl * kPl + off) = make_uint4(pc[pl][0], pc[pl][1], pc[pl][2], pc[pl][3]);
  }
}

// TF32 operands are read K-major only: elements (c..c+3, r) of the float32 plane.
template <int C = 128>
__device__ __forceinline__ void store4_t(uint8_t* base, int r, int c, float4 v, float s) {
  *(float*)(base + op_off<PMF_PREC_TF32, C>(c + 0, r)) = v.x * s;
  *(float*)(base + op_off<PMF_PREC_TF32, C>(c + 1, r)) = v.y * s;
  *(float*)(base + op_off<PMF_PREC_TF32, C>(c + 2, r)) = v.z * s;
  *(float*)(base + op_off<PMF_PREC_TF32, C>(c + 3, r)) = v.w * s;
}

__device__ __forceinline__ float amax4(float m, float4 v) {
  return fmaxf(fmaxf(m, fmaxf(fabsf(v.x), fabsf(v.y))), fmaxf(fabsf(v.z), fabsf(v.w)));
}

// Power-of-two scale bringing max |v| to [2^13, 2^14) for FP16 operands; 1 otherwise.
// The exponent is capped at 2^100 so that the scale and the product with the
// matrix scale (2^14) stay finite when a tile holds only tiny or denormal
// values (e.g. a 3-D slice far from the mass).
template <int P>
__device__ __forceinline__ float op_scale(float mx) {
  if (P != PMF_PREC_FP16X3 || !(mx > 0.0f) || !isfinite(mx)) return 1.0f;
  int e;
  frexpf(mx, &e);
  return ldexpf(1.0f, min(14 - e, 100));
}


// Double-float (hi + lo float32 pair) arithmetic: float64-class accuracy for
// the moment sums at float32 throughput (GB300 issues float64 at ~1/32 of the
// float32 rate, so block-wide float64 reductions are avoided).
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const float s = a.hi + b.hi;
  const float bb = s - a.hi;
  const float e = (a.hi - (s - bb)) + (b.hi - bb);
  const float t = e + a.lo + b.lo;
  const float h = s + t;
  return DF{h, t - (h - s)};
}
__device__ __forceinline__ DF df_add1(DF a, float b) { return df_add(a, DF{b, 0.0f}); }

// Moment sums of one thread: S0, S1 (u0, u1), S2 (u0u0, u0u1, u1u1).  Points
// arrive in groups (a thread's row segment, or a thread's four columns); the
// group sums are formed in float32 (at most ~40 terms) and added in
// double-float.
struct Moments {
  DF s[6];
  __device__ __forceinline__ void zero() {
#pragma unroll
    for (int i = 0; i < 6; ++i) s[i] = DF{0.0f, 0.0f};
  }
  // float32 sums of a row segment at u0: a = sum x, b = sum x u1, c = sum x u1^2
  __device__ __forceinline__ void add_row(float a, float b, float c, float u0) {
    s[0] = df_add1(s[0], a);
    s[1] = df_add1(s[1], a * u0);
    s[2] = df_add1(s[2], b);
    s[3] = df_add1(s[3], a * u0 * u0);
    s[4] = df_add1(s[4], b * u0);
    s[5] = df_add1(s[5], c);
  }
  // float32 sums of four columns u1 + 0..3: a[i] = sum x, b[i] = sum x u0,
  // c[i] = sum x u0^2 over the rows of column i
  __device__ __forceinline__ void add_cols4(const float* a, const float* b, const float* c, float u1) {
    float s0 = 0.0f, s1 = 0.0f, s2 = 0.0f, s3 = 0.0f, s4 = 0.0f, s5 = 0.0f;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const float v = u1 + (float)i;
      s0 += a[i];
      s1 += b[i];
      s2 = fmaf(a[i], v, s2);
      s3 += c[i];
      s4 = fmaf(b[i], v, s4);
      s5 = fmaf(a[i] * v, v, s5);
    }
    s[0] = df_add1(s[0], s0);
    s[1] = df_add1(s[1], s1);
    s[2] = df_add1(s[2], s2);
    s[3] = df_add1(s[3], s3);
    s[4] = df_add1(s[4], s4);
    s[5] = df_add1(s[5], s5);
  }
};

// Issue one GEMM stage (one thread): D = A * W^T, A read K-major or MN-major.
// For the split formats the correction products are accumulated first, while
// the FP32 accumulator is small, and the hi*hi products last, so that only
// those see roundings at full magnitude: hi*lo, lo*hi (~2^-11 of the result)
// for the two-piece formats; for BF16X6 (pieces hi, mid, lo of ~2^0, 2^-9,
// 2^-18) hi*lo, lo*hi and mid*mid (~2^-18), then hi*mid and mid*hi (~2^-9).
template <int P, int C = 128, int R = 128>
__device__ __forceinline__ void issue_stage(uint32_t tmem, uint32_t a_base, int a_mn, uint32_t w_base,
                                            int nout, int K, uint32_t mbar) {
  constexpr uint32_t rb = Lay<P, C>::rowblk;
  constexpr uint32_t kPl = Lay<P, C, R>::plane, kWPl = Lay<P, C>::wplane;
  constexpr int kp = Fmt<P>::kper;
  const uint32_t id = idesc(Fmt<P>::code, a_mn, nout);
  // K step of one instruction: 32 bytes = 2 core matrices along K (K-major),
  // or kp rows = kp/8 row blocks (MN-major)
  auto adesc = [&](uint32_t base, int ks) {
    return a_mn ? sdesc(base + ks * (kp / 8) * rb, rb, 128) : sdesc(base + ks * 256, 128, rb);
  };
  if constexpr (Fmt<P>::planes == 1) {
    for (int ks = 0; ks < K / kp; ++ks)
      mma_tf32(tmem, adesc(a_base, ks), sdesc(w_base + ks * 256, 128, rb), id, ks > 0);
  } else if constexpr (Fmt<P>::planes == 3) {
    for (int ks = 0; ks < K / kp; ++ks) {
      mma_f16(tmem, adesc(a_base, ks), sdesc(w_base + 2 * kWPl + ks * 256, 128, rb), id, ks > 0);
      mma_f16(tmem, adesc(a_base + 2 * kPl, ks), sdesc(w_base + ks * 256, 128, rb), id, 1);
      mma_f16(tmem, adesc(a_base + kPl, ks), sdesc(w_base + kWPl + ks * 256, 128, rb), id, 1);
    }
    for (int ks = 0; ks < K / kp; ++ks) {
      mma_f16(tmem, adesc(a_base, ks), sdesc(w_base + kWPl + ks * 256, 128, rb), id, 1);
      mma_f16(tmem, adesc(a_base + kPl, ks), sdesc(w_base + ks * 256, 128, rb), id, 1);
    }
    for (int ks = 0; ks < K / kp; ++ks)
      mma_f16(tmem, adesc(a_base, ks), sdesc(w_base + ks * 256, 128, rb), id, 1);
  } else {
    for (int ks = 0; ks < K / kp; ++ks) {
      mma_f16(tmem, adesc(a_base, ks), sdesc(w_base + kWPl + ks * 256, 128, rb), id, ks > 0);
      mma_f16(tmem, adesc(a_base + kPl, ks), sdesc(w_base + ks * 256, 128, rb), id, 1);
    }
    for (int ks = 0; ks < K / kp; ++ks)
      mma_f16(tmem, adesc(a_base, ks), sdesc(w_base + ks * 256, 128, rb), id, 1);
  }
  mma_commit(mbar);
}

// Row parameters of the separable regrid along one axis (float64 per row):
// y_n = rs + rd u_n, z_n = y_n + (N-1)/2 = i_n + f_n with |f_n| <= 1/2.
template <int R>
struct RegridRowsT {
  int ri[R];
  float rf[R], rS[R], rcf[R], rsf[R];
  unsigned char rzero[R];
};
using RegridRows = RegridRowsT<128>;

template <int R>
__device__ void regrid_rows(RegridRowsT<R>& sh, double rs, double rd, int N, int t0, int tstep) {
  for (int n = t0; n < N; n += tstep) {
    const double y = rs + rd * (n - 0.5 * (N - 1));
    const double z = y + 0.5 * (N - 1);
    const double i = rint(fmin(fmax(z, -1.0), (double)N + 1.0));
    const float f = (float)(z - i);
    sh.ri[n] = (int)i;
    sh.rf[n] = f;
    sh.rzero[n] = !(fabs(y) <= 0.5 * N);  // also zero (and skip the table) for a non-finite y
    sh.rS[n] = sinpif(f);
    float s, c;
    sincospif(f / (float)N, &s, &c);
    sh.rsf[n] = s;
    sh.rcf[n] = c;
  }
}

// Entry (n, j) of the periodic-sinc regrid matrix (rows: new nodes, columns:
// old nodes): I[n, j] = sin(pi v) / (N tan(pi v / N)), v = y_n - u_j = m + f_n,
// m = i_n - j, evaluated as (-1)^m sin(pi f) cos(pi v/N) / (N sin(pi v/N)) with
// the angle pi v / N split into the tabulated pi m / N (sctab: (cos, sin) for
// m = -N..N) and the per-row pi f / N.  Rows of new nodes outside the old box
// are zero.
struct RegridRow {
  int i;
  float f, S, cf, sf;
  bool zero;
};

template <int R>
__device__ __forceinline__ RegridRow regrid_row(const RegridRowsT<R>& sh, int n) {
  return RegridRow{sh.ri[n], sh.rf[n], sh.rS[n], sh.rcf[n], sh.rsf[n], sh.rzero[n] != 0};
}

__device__ __forceinline__ float interp_value(const RegridRow& r, int j, int N, const float* sctab) {
  if (r.zero) return 0.0f;
  const int m = r.i - j;
  if (m == 0 && r.f == 0.0f) return 1.0f;
  const float cm = sctab[2 * (m + N)], sm = sctab[2 * (m + N) + 1];
  const float sv = sm * r.cf + cm * r.sf;
  const float cv = cm * r.cf - sm * r.sf;
  return __fdividef(((m & 1) ? -1.0f : 1.0f) * r.S * cv, (float)N * sv);
}

template <int R>
__device__ __forceinline__ float interp_entry(const RegridRowsT<R>& sh, int n, int j, int N, const float* sctab) {
  return interp_value(regrid_row(sh, n), j, N, sctab);
}

// The regrid matrix of one axis into the W planes, scaled by sw (identity
// when the frame was re-aligned: the gather already moved the weights).
// Thread t0 (of tstep >= N) keeps row t0 % N and every (tstep / N)-th group
// of four columns, so its row parameters are read once; consecutive threads
// take consecutive rows (8 rows share 128 bytes of the operand layout).
template <int P, int C = 128, int R = 128>
__device__ void build_interp(const RegridRowsT<R>& sh, uint8_t* W, int N, const float* sctab, float sw, int realign,
                             int t0, int tstep) {
  const int per = tstep / N;
  if (t0 >= per * N) return;
  const int n = t0 % N;
  const RegridRow r = regrid_row(sh, n);
  for (int c = (t0 / N) * 8; c < N; c += 8 * per) {   // N is a multiple of 16
    float k[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int j = c + i;
      k[i] = realign ? (n == j ? 1.0f : 0.0f) : interp_value(r, j, N, sctab);
    }
    store8<P, C, true>(W, n, c, make_float4(k[0], k[1], k[2], k[3]), make_float4(k[4], k[5], k[6], k[7]), sw);
  }
}

}  // namespace
}  // namespace pmf
