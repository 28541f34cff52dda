// fp32 GEMM on the 5th-generation tensor cores with a three-term tf32 split:
//     Y[M, N] = act(X[M, K] W[N, K]^T + b)
// x = x_hi + x_lo with x_hi = tf32(x) (round to nearest) and x_lo = x - x_hi
// (exact in fp32), likewise for W; the product is accumulated in fp32 tensor
// memory as x_hi w_hi + x_hi w_lo + x_lo w_hi.  The dropped x_lo w_lo term and
// the tf32 rounding of the lo parts are each below 2^-22 of |x||w|, so every
// output is within about 3 * 2^-22 * sum_k |x_k||w_k| of the exact dot product
// -- fp32-level accuracy at tensor-core speed.
//
// One CTA computes a 128 x BN tile with 6 warps:
//   warp 0, one lane : TMA producer, 128x32 fp32 tiles of X and BNx32 of W
//                      (128-byte swizzle) into a STAGES-deep ring;
//   warps 2-5        : splitters -- per stage, rewrite each loaded tile in place
//                      as its tf32 hi part and write its lo part to a twin buffer
//                      (same swizzled layout), then fence for the async proxy;
//   warp 1, one lane : MMA issuer -- per 8-wide k-step three tcgen05.mma
//                      kind::tf32 into a 128 x BN fp32 TMEM accumulator;
//   warps 2-5        : epilogue -- tcgen05.ld of 32 TMEM lanes each, bias, ReLU,
//                      fp32 16-byte stores.
// Each output's k order is fixed, so a row's result does not depend on M.
#include <algorithm>

#include "kernels.h"

namespace sage {
namespace {

constexpr int kBM = 128, kBK = 32;  // 32 fp32 = one 128-byte swizzle row

template <int BN, int NST>
struct Tf32Cfg {
  static constexpr int A_BYTES = kBM * kBK * 4;  // 16 KB
  static constexpr int B_BYTES = BN * kBK * 4;
  static constexpr int STAGE = 2 * (A_BYTES + B_BYTES);  // hi + lo of both operands
  static constexpr int STAGES = NST;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 512;
  static_assert(STAGES >= 2, "pipeline depth");
};

constexpr int kSplitThreads = 128;  // warps 2..5

// In place: v -> tf32(v); lo buffer: v - tf32(v).  `n4` float4 per thread-stride pass.
__device__ __forceinline__ void split_tile(float* hi, float* lo, int nfloat, int tid) {
  float4* h4 = reinterpret_cast<float4*>(hi);
  float4* l4 = reinterpret_cast<float4*>(lo);
  for (int q = tid; q < nfloat / 4; q += kSplitThreads) {
    const float4 v = h4[q];
    float4 h, l;
    h.x = to_tf32_rna(v.x);
    h.y = to_tf32_rna(v.y);
    h.z = to_tf32_rna(v.z);
    h.w = to_tf32_rna(v.w);
    l.x = v.x - h.x;
    l.y = v.y - h.y;
    l.z = v.z - h.z;
    l.w = v.w - h.w;
    h4[q] = h;
    l4[q] = l;
  }
}

template <int BN, int NST>
__global__ void __launch_bounds__(192, 1)
    gemm_tf32x3_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M,
                       int N, int K, const float* __restrict__ bias, int relu, float* __restrict__ Y, int ldy,
                       int* err) {
  using C = Tf32Cfg<BN, NST>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  // per stage: A_hi | B_hi | A_lo | B_lo
  auto a_hi = [&](int s) { return smem + s * C::STAGE; };
  auto b_hi = [&](int s) { return smem + s * C::STAGE + C::A_BYTES; };
  auto a_lo = [&](int s) { return smem + s * C::STAGE + C::A_BYTES + C::B_BYTES; };
  auto b_lo = [&](int s) { return smem + s * C::STAGE + 2 * C::A_BYTES + C::B_BYTES; };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  uint64_t* split = full + C::STAGES;
  uint64_t* empty = split + C::STAGES;
  uint64_t* accum = empty + C::STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * kBM;
  const int KB = (K + kBK - 1) / kBK;

  if (warp == 0) tmem_alloc(tmem_slot, BN);
  if (warp == 1 && lane == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&split[s], kSplitThreads);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    fence_mbar_init();
  }
  if (warp == 2 && lane == 0) {
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      // ---- TMA producer
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % C::STAGES;
        const uint32_t ph = (kb / C::STAGES) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, err)) break;
        mbar_arrive_expect_tx(&full[s], C::A_BYTES + C::B_BYTES);
        tma_load_2d(a_hi(s), &tmA, kb * kBK, m0, &full[s]);
        tma_load_2d(b_hi(s), &tmB, kb * kBK, n0, &full[s]);
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      // ---- MMA issuer: hi*hi + hi*lo + lo*hi per 8-wide k-step
      constexpr uint32_t idesc = idesc_tf32_f32(kBM, BN);
      for (int kb = 0; kb < KB; ++kb) {
        const int s = kb % C::STAGES;
        const uint32_t ph = (kb / C::STAGES) & 1;
        if (!mbar_wait(&split[s], ph, err)) break;
        tc_fence_after();
        const uint32_t ah = smem_u32(a_hi(s)), bh = smem_u32(b_hi(s));
        const uint32_t al = smem_u32(a_lo(s)), bl = smem_u32(b_lo(s));
#pragma unroll
        for (int k = 0; k < kBK / 8; ++k) {
          const uint32_t o = k * 32;  // 8 fp32 = 32 bytes along K inside the swizzle row
          tc_mma_tf32_fill_a(tmem, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bh + o), idesc,
                             (kb | k) != 0 ? 1u : 0u);
          tc_mma_tf32_lastuse_a(tmem, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bl + o), idesc, 1u);
          tc_mma_tf32(tmem, sw128_kmajor_desc(al + o), sw128_kmajor_desc(bh + o), idesc, 1u);
        }
        tc_commit(&empty[s]);
      }
      tc_commit(accum);
    }
  } else {
    // ---- splitters
    const int tid = threadIdx.x - 64;
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (kb / C::STAGES) & 1;
      if (!mbar_wait(&full[s], ph, err)) break;
      split_tile(reinterpret_cast<float*>(a_hi(s)), reinterpret_cast<float*>(a_lo(s)), kBM * kBK, tid);
      split_tile(reinterpret_cast<float*>(b_hi(s)), reinterpret_cast<float*>(b_lo(s)), BN * kBK, tid);
      fence_proxy_async_smem();
      mbar_arrive(&split[s]);
    }
  }
  __syncwarp();

  // ---- epilogue (warps 2-5; warp w reads TMEM lanes 32*(w%4) .. +31)
  if (warp >= 2) {
    mbar_wait(accum, 0, err);
    tc_fence_after();
    const int q = warp & 3;
    const int row = m0 + q * 32 + lane;
    float* yrow = Y + static_cast<size_t>(row < M ? row : 0) * ldy + n0;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 32) {
      uint32_t v[32];
      tmem_ld_32cols(tmem + (static_cast<uint32_t>(q * 32) << 16) + c0, v);
      tmem_ld_wait();
      if (row < M) {
        float4* dst = reinterpret_cast<float4*>(yrow + c0);
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          float4 o;
          o.x = __uint_as_float(v[4 * j + 0]) + __ldg(bias + n0 + c0 + 4 * j + 0);
          o.y = __uint_as_float(v[4 * j + 1]) + __ldg(bias + n0 + c0 + 4 * j + 1);
          o.z = __uint_as_float(v[4 * j + 2]) + __ldg(bias + n0 + c0 + 4 * j + 2);
          o.w = __uint_as_float(v[4 * j + 3]) + __ldg(bias + n0 + c0 + 4 * j + 3);
          if (relu) {
            o.x = fmaxf(o.x, 0.f);
            o.y = fmaxf(o.y, 0.f);
            o.z = fmaxf(o.z, 0.f);
            o.w = fmaxf(o.w, 0.f);
          }
          dst[j] = o;
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// Pre-split operands: X and W arrive as hi/lo planes (x = hi + lo, hi = tf32(x)),
// so the pipeline is TMA -> MMA only (4 warps: warp 0 lane 0 loads the four
// tiles of a stage, warp 1 lane 0 issues the MMAs, all four warps run the
// epilogue).  The epilogue writes the output as hi/lo planes too, ready for the
// next layer.  Same products in the same order as the splitting kernel above,
// so the results are bitwise the same.
template <int BN, int NST>
__global__ void __launch_bounds__(128, 1)
    gemm_tf32x3_presplit_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                                const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                                int M, int N, int K, const float* __restrict__ bias, int relu,
                                float* __restrict__ Yh, float* __restrict__ Yl, int ldy, int* err) {
  using C = Tf32Cfg<BN, NST>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  auto a_hi = [&](int s) { return smem + s * C::STAGE; };
  auto b_hi = [&](int s) { return smem + s * C::STAGE + C::A_BYTES; };
  auto a_lo = [&](int s) { return smem + s * C::STAGE + C::A_BYTES + C::B_BYTES; };
  auto b_lo = [&](int s) { return smem + s * C::STAGE + 2 * C::A_BYTES + C::B_BYTES; };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* accum = empty + C::STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accum + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n0 = blockIdx.x * BN, m0 = blockIdx.y * kBM;
  const int KB = (K + kBK - 1) / kBK;

  if (warp == 0) tmem_alloc(tmem_slot, BN);
  if (warp == 1 && lane == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accum, 1);
    fence_mbar_init();
  }
  if (warp == 2 && lane == 0) {
    tma_prefetch_desc(&tmAh);
    tma_prefetch_desc(&tmAl);
    tma_prefetch_desc(&tmBh);
    tma_prefetch_desc(&tmBl);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (kb / C::STAGES) & 1;
      if (!mbar_wait(&empty[s], ph ^ 1, err)) break;
      mbar_arrive_expect_tx(&full[s], C::STAGE);
      tma_load_2d(a_hi(s), &tmAh, kb * kBK, m0, &full[s]);
      tma_load_2d(a_lo(s), &tmAl, kb * kBK, m0, &full[s]);
      tma_load_2d(b_hi(s), &tmBh, kb * kBK, n0, &full[s]);
      tma_load_2d(b_lo(s), &tmBl, kb * kBK, n0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = idesc_tf32_f32(kBM, BN);
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (kb / C::STAGES) & 1;
      if (!mbar_wait(&full[s], ph, err)) break;
      tc_fence_after();
      const uint32_t ah = smem_u32(a_hi(s)), bh = smem_u32(b_hi(s));
      const uint32_t al = smem_u32(a_lo(s)), bl = smem_u32(b_lo(s));
#pragma unroll
      for (int k = 0; k < kBK / 8; ++k) {
        const uint32_t o = k * 32;
        tc_mma_tf32_fill_a(tmem, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bh + o), idesc,
                           (kb | k) != 0 ? 1u : 0u);
        tc_mma_tf32_lastuse_a(tmem, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bl + o), idesc, 1u);
        tc_mma_tf32(tmem, sw128_kmajor_desc(al + o), sw128_kmajor_desc(bh + o), idesc, 1u);
      }
      tc_commit(&empty[s]);
    }
    tc_commit(accum);
  }
  __syncwarp();

  mbar_wait(accum, 0, err);
  tc_fence_after();
  const int row = m0 + warp * 32 + lane;
  const size_t ro = static_cast<size_t>(row < M ? row : 0) * ldy + n0;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t v[32];
    tmem_ld_32cols(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
    tmem_ld_wait();
    if (row < M) {
      float4* dh = reinterpret_cast<float4*>(Yh + ro + c0);
      float4* dl = reinterpret_cast<float4*>(Yl + ro + c0);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        float o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          o[q] = __uint_as_float(v[4 * j + q]) + __ldg(bias + n0 + c0 + 4 * j + q);
          if (relu) o[q] = fmaxf(o[q], 0.f);
        }
        float4 h, l;
        h.x = to_tf32_rna(o[0]);
        h.y = to_tf32_rna(o[1]);
        h.z = to_tf32_rna(o[2]);
        h.w = to_tf32_rna(o[3]);
        l.x = o[0] - h.x;
        l.y = o[1] - h.y;
        l.z = o[2] - h.z;
        l.w = o[3] - h.w;
        dh[j] = h;
        dl[j] = l;
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// Persistent form of the pre-split kernel: one CTA per SM walks the output tiles
// (n fastest, so neighbouring CTAs share X tiles in L2).  Two TMEM accumulators
// alternate between tiles, so the epilogue warps drain tile i while the MMA warp
// computes tile i+1; the shared-memory ring runs on across tile boundaries.
//   warp 0 lane 0: TMA producer; warp 1 lane 0: MMA issuer;
//   warps 2-5: epilogue (warp w reads TMEM lanes 32*(w%4)..+31).
// With HEAD the epilogue writes no Y: it fuses the sigmoid head (HeadParams).
// Without HEAD, when the last wave of tiles would leave more than half of the CTAs
// idle, its tiles run as two half-width items each (B maps tmBh2 / tmBl2, boxes of
// BN / 2 rows), so that wave takes half as long; the MMAs per output element are the
// same, so are the bits.
template <int BN, int NST, bool HEAD>
__device__ __forceinline__ void tf32x3_persistent_body(const CUtensorMap& tmAh, const CUtensorMap& tmAl,
                                                       const CUtensorMap& tmBh, const CUtensorMap& tmBl, int M,
                                                       int N, int K, const float* __restrict__ bias, int relu,
                                                       float* __restrict__ Yh, float* __restrict__ Yl, int ldy,
                                                       int* err, const HeadParams* hp, const CUtensorMap* tmYh,
                                                       const CUtensorMap* tmYl, const CUtensorMap* tmBh2 = nullptr,
                                                       const CUtensorMap* tmBl2 = nullptr) {
  using C = Tf32Cfg<BN, NST>;
  static_assert(HEAD || C::STAGES * C::STAGE >= 4 * 32768, "last-tile output staging: 32 KB per epilogue warp");
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_align1024(smem_raw);
  auto a_hi = [&](int s) { return smem + s * C::STAGE; };
  auto b_hi = [&](int s) { return smem + s * C::STAGE + C::A_BYTES; };
  auto a_lo = [&](int s) { return smem + s * C::STAGE + C::A_BYTES + C::B_BYTES; };
  auto b_lo = [&](int s) { return smem + s * C::STAGE + 2 * C::A_BYTES + C::B_BYTES; };
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + C::STAGES * C::STAGE);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;  // [2]
  uint64_t* acc_empty = acc_full + 2;      // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = (K + kBK - 1) / kBK;
  const int NT = N / BN, MT = (M + kBM - 1) / kBM;
  const int tiles = NT * MT;
  // work items: tiles, the last wave's split in halves when that halves its time
  const int GR = static_cast<int>(gridDim.x);
  int nfull = tiles, items = tiles;
  if (!HEAD && tmBh2 && tiles > GR && tiles % GR != 0 && 2 * (tiles % GR) <= GR) {
    nfull = tiles - tiles % GR;
    items = nfull + 2 * (tiles % GR);
  }
  auto item = [&](int w, int& m0, int& n0, int& width) {
    if (w < nfull) {
      m0 = (w / NT) * kBM;
      n0 = (w % NT) * BN;
      width = BN;
    } else {
      const int h = w - nfull, t = nfull + h / 2;
      m0 = (t / NT) * kBM;
      n0 = (t % NT) * BN + (h & 1) * (BN / 2);
      width = BN / 2;
    }
  };

  if (warp == 0) tmem_alloc(tmem_slot, 2 * BN);
  if (warp == 1 && lane == 0) {
    for (int s = 0; s < C::STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    fence_mbar_init();
  }
  if (warp == 2 && lane == 0) {
    tma_prefetch_desc(&tmAh);
    tma_prefetch_desc(&tmAl);
    tma_prefetch_desc(&tmBh);
    tma_prefetch_desc(&tmBl);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;  // stage use counter across tiles
      bool ok = true;
      for (int w = blockIdx.x; w < items && ok; w += gridDim.x) {
        int m0, n0, width;
        item(w, m0, n0, width);
        const bool whole = width == BN;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % C::STAGES;
          const uint32_t ph = (g / C::STAGES) & 1;
          if (!mbar_wait(&empty[s], ph ^ 1, err)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], whole ? C::STAGE : C::STAGE - C::B_BYTES);
          tma_load_2d(a_hi(s), &tmAh, kb * kBK, m0, &full[s]);
          tma_load_2d(a_lo(s), &tmAl, kb * kBK, m0, &full[s]);
          tma_load_2d(b_hi(s), whole ? &tmBh : tmBh2, kb * kBK, n0, &full[s]);
          tma_load_2d(b_lo(s), whole ? &tmBl : tmBl2, kb * kBK, n0, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc_whole = idesc_tf32_f32(kBM, BN), idesc_half = idesc_tf32_f32(kBM, BN / 2);
      uint32_t g = 0;
      int i = 0;
      bool ok = true;
      for (int w = blockIdx.x; w < items && ok; w += gridDim.x, ++i) {
        const uint32_t idesc = w < nfull ? idesc_whole : idesc_half;
        const int buf = i & 1;
        const uint32_t acc = tmem + static_cast<uint32_t>(buf * BN);
        if (!mbar_wait(&acc_empty[buf], ((i >> 1) & 1) ^ 1, err)) break;
        tc_fence_after();
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % C::STAGES;
          const uint32_t ph = (g / C::STAGES) & 1;
          if (!mbar_wait(&full[s], ph, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = smem_u32(a_hi(s)), bh = smem_u32(b_hi(s));
          const uint32_t al = smem_u32(a_lo(s)), bl = smem_u32(b_lo(s));
#pragma unroll
          for (int k = 0; k < kBK / 8; ++k) {
            const uint32_t o = k * 32;
            tc_mma_tf32_fill_a(acc, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bh + o), idesc,
                               (kb | k) != 0 ? 1u : 0u);
            tc_mma_tf32_lastuse_a(acc, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bl + o), idesc, 1u);
            tc_mma_tf32(acc, sw128_kmajor_desc(al + o), sw128_kmajor_desc(bh + o), idesc, 1u);
          }
          tc_commit(&empty[s]);
        }
        tc_commit(&acc_full[buf]);
      }
    }
  } else {
    // ---- epilogue warps
    const int q = warp & 3;
    int i = 0;
    for (int w = blockIdx.x; w < items; w += gridDim.x, ++i) {
      const int buf = i & 1;
      int m0, n0, width;
      item(w, m0, n0, width);
      if (!mbar_wait(&acc_full[buf], (i >> 1) & 1, err)) break;
      tc_fence_after();
      const int row = m0 + q * 32 + lane;
      if constexpr (HEAD) {
        // group sums of the head's products, then release the accumulator
        const unsigned G = static_cast<unsigned>(N / 64);
        const float* hw = static_cast<const float*>(hp->f.w) + n0;
        float gs[BN / 64];
#pragma unroll
        for (int c0 = 0; c0 < BN; c0 += 64) {
          float gsum = 0.f;
#pragma unroll
          for (int half = 0; half < 2; ++half) {
            uint32_t v[32];
            tmem_ld_32cols(tmem + static_cast<uint32_t>(buf * BN) + (static_cast<uint32_t>(q * 32) << 16) + c0 +
                               32 * half,
                           v);
            tmem_ld_wait();
            float p[32];
#pragma unroll
            for (int j = 0; j < 32; ++j) {
              float o = __uint_as_float(v[j]) + __ldg(bias + n0 + c0 + 32 * half + j);
              if (relu) o = fmaxf(o, 0.f);
              p[j] = __fmul_rn(o, __ldg(hw + c0 + 32 * half + j));
            }
            const float ch = head_tree32(p);
            gsum = half == 0 ? ch : __fadd_rn(gsum, ch);
          }
          gs[c0 / 64] = gsum;
        }
        tc_fence_before();
        mbar_arrive(&acc_empty[buf]);
        if (row < M) head_row<BN / 64>(*hp, row, gs, static_cast<unsigned>(n0 / 64), G);
        continue;
      }
      if (w + static_cast<int>(gridDim.x) >= items) {
        // the CTA's last tile: out through the idle stage ring and TMA stores
        tail_store_f32_planes<BN, 4>(tmem + static_cast<uint32_t>(buf * BN) + (static_cast<uint32_t>(q * 32) << 16),
                                  smem + q * 32768, lane, bias, relu != 0, tmYh, tmYl, n0, m0 + q * 32,
                                  m0 + q * 32 < M, 0, 1, width);
        tc_fence_before();
        mbar_arrive(&acc_empty[buf]);
        continue;
      }
      const size_t ro = static_cast<size_t>(row < M ? row : 0) * ldy + n0;
#pragma unroll 1
      for (int c0 = 0; c0 < width; c0 += 32) {
        uint32_t v[32];
        tmem_ld_32cols(tmem + static_cast<uint32_t>(buf * BN) + (static_cast<uint32_t>(q * 32) << 16) + c0, v);
        tmem_ld_wait();
        if (row < M) {
          float4* dh = reinterpret_cast<float4*>(Yh + ro + c0);
          float4* dl = reinterpret_cast<float4*>(Yl + ro + c0);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              o[u] = __uint_as_float(v[4 * j + u]) + __ldg(bias + n0 + c0 + 4 * j + u);
              if (relu) o[u] = fmaxf(o[u], 0.f);
            }
            float4 h, l;
            h.x = to_tf32_rna(o[0]);
            h.y = to_tf32_rna(o[1]);
            h.z = to_tf32_rna(o[2]);
            h.w = to_tf32_rna(o[3]);
            l.x = o[0] - h.x;
            l.y = o[1] - h.y;
            l.z = o[2] - h.z;
            l.w = o[3] - h.w;
            dh[j] = h;
            dl[j] = l;
          }
        }
      }
      // this thread's TMEM reads of `buf` are complete: hand the buffer back to the MMA warp
      tc_fence_before();
      mbar_arrive(&acc_empty[buf]);
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * BN);
}

template <int BN, int NST>
__global__ void __launch_bounds__(192, 1)
    gemm_tf32x3_persistent_kernel(const __grid_constant__ CUtensorMap tmAh, const __grid_constant__ CUtensorMap tmAl,
                                  const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                                  const __grid_constant__ CUtensorMap tmYh, const __grid_constant__ CUtensorMap tmYl,
                                  const __grid_constant__ CUtensorMap tmBh2, const __grid_constant__ CUtensorMap tmBl2,
                                  int M, int N, int K, const float* __restrict__ bias, int relu,
                                  float* __restrict__ Yh, float* __restrict__ Yl, int ldy, int* err) {
  tf32x3_persistent_body<BN, NST, false>(tmAh, tmAl, tmBh, tmBl, M, N, K, bias, relu, Yh, Yl, ldy, err, nullptr,
                                         &tmYh, &tmYl, &tmBh2, &tmBl2);
}

template <int BN, int NST>
__global__ void __launch_bounds__(192, 1)
    gemm_tf32x3_persistent_head_kernel(const __grid_constant__ CUtensorMap tmAh,
                                       const __grid_constant__ CUtensorMap tmAl,
                                       const __grid_constant__ CUtensorMap tmBh,
                                       const __grid_constant__ CUtensorMap tmBl, int M, int N, int K,
                                       const float* __restrict__ bias, int relu, int* err,
                                       const __grid_constant__ HeadParams hp) {
  tf32x3_persistent_body<BN, NST, true>(tmAh, tmAl, tmBh, tmBl, M, N, K, bias, relu, nullptr, nullptr, 0, err, &hp,
                                        nullptr, nullptr);
}

__global__ void split_planes_kernel(const float* __restrict__ src, float* __restrict__ hi, float* __restrict__ lo,
                                    size_t n) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    const float v = src[i];
    const float h = to_tf32_rna(v);
    hi[i] = h;
    lo[i] = v - h;
  }
}

template <int BN, int NST>
cudaError_t launch_presplit_bn(int M, int N, int K, const float* xh, const float* xl, int ldx, const float* wh,
                               const float* wl, const float* bias, int relu, float* yh, float* yl, int ldy, int* err,
                               cudaStream_t s) {
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(gemm_tf32x3_presplit_kernel<BN, NST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, Tf32Cfg<BN, NST>::SMEM);
      });
      e != cudaSuccess)
    return e;
  CUtensorMap tah, tal, tbh, tbl;
  if (!make_tmap_2d(&tah, 0, xh, M, K, ldx, kBK, kBM) || !make_tmap_2d(&tal, 0, xl, M, K, ldx, kBK, kBM) ||
      !make_tmap_2d(&tbh, 0, wh, N, K, K, kBK, BN) || !make_tmap_2d(&tbl, 0, wl, N, K, K, kBK, BN))
    return cudaErrorInvalidValue;
  dim3 grid(N / BN, (M + kBM - 1) / kBM);
  gemm_tf32x3_presplit_kernel<BN, NST><<<grid, 128, Tf32Cfg<BN, NST>::SMEM, s>>>(tah, tal, tbh, tbl, M, N, K, bias,
                                                                                 relu, yh, yl, ldy, err);
  count_launch();
  return cudaGetLastError();
}

template <int BN, int NST>
cudaError_t launch_persistent_bn(int M, int N, int K, const float* xh, const float* xl, int ldx, const float* wh,
                                 const float* wl, const float* bias, int relu, float* yh, float* yl, int ldy,
                                 int* err, cudaStream_t s) {
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(gemm_tf32x3_persistent_kernel<BN, NST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, Tf32Cfg<BN, NST>::SMEM);
      });
      e != cudaSuccess)
    return e;
  CUtensorMap tah, tal, tbh, tbl, tyh, tyl, tbh2, tbl2;
  if (!make_tmap_2d(&tah, 0, xh, M, K, ldx, kBK, kBM) || !make_tmap_2d(&tal, 0, xl, M, K, ldx, kBK, kBM) ||
      !make_tmap_2d(&tbh, 0, wh, N, K, K, kBK, BN) || !make_tmap_2d(&tbl, 0, wl, N, K, K, kBK, BN) ||
      !make_tmap_2d(&tbh2, 0, wh, N, K, K, kBK, BN / 2) || !make_tmap_2d(&tbl2, 0, wl, N, K, K, kBK, BN / 2) ||
      !make_tmap_2d(&tyh, 0, yh, M, N, ldy, 32, 32) || !make_tmap_2d(&tyl, 0, yl, M, N, ldy, 32, 32))
    return cudaErrorInvalidValue;
  const int tiles = (N / BN) * ((M + kBM - 1) / kBM);
  const int sms_n = device_sms();
  const int grid = tiles < sms_n ? tiles : sms_n;
  gemm_tf32x3_persistent_kernel<BN, NST><<<grid, 192, Tf32Cfg<BN, NST>::SMEM, s>>>(
      tah, tal, tbh, tbl, tyh, tyl, tbh2, tbl2, M, N, K, bias, relu, yh, yl, ldy, err);
  count_launch();
  return cudaGetLastError();
}

template <int BN, int NST>
cudaError_t launch_persistent_head_bn(int M, int N, int K, const float* xh, const float* xl, int ldx,
                                      const float* wh, const float* wl, const float* bias, int relu, int* err,
                                      cudaStream_t s, const HeadParams& hp) {
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(gemm_tf32x3_persistent_head_kernel<BN, NST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, Tf32Cfg<BN, NST>::SMEM);
      });
      e != cudaSuccess)
    return e;
  CUtensorMap tah, tal, tbh, tbl;
  if (!make_tmap_2d(&tah, 0, xh, M, K, ldx, kBK, kBM) || !make_tmap_2d(&tal, 0, xl, M, K, ldx, kBK, kBM) ||
      !make_tmap_2d(&tbh, 0, wh, N, K, K, kBK, BN) || !make_tmap_2d(&tbl, 0, wl, N, K, K, kBK, BN))
    return cudaErrorInvalidValue;
  const int tiles = (N / BN) * ((M + kBM - 1) / kBM);
  const int sms_n = device_sms();
  const int grid = tiles < sms_n ? tiles : sms_n;
  gemm_tf32x3_persistent_head_kernel<BN, NST><<<grid, 192, Tf32Cfg<BN, NST>::SMEM, s>>>(
      tah, tal, tbh, tbl, M, N, K, bias, relu, err, hp);
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_presplit_cfg(GemmCfg c, int M, int N, int K, const float* xh, const float* xl, int ldx,
                                const float* wh, const float* wl, const float* bias, int relu, float* yh, float* yl,
                                int ldy, int* err, cudaStream_t s) {
  if (c.bn == 128 && c.stages == 3)
    return launch_presplit_bn<128, 3>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, yh, yl, ldy, err, s);
  if (c.bn == 64 && c.stages == 4)
    return launch_presplit_bn<64, 4>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, yh, yl, ldy, err, s);
  if (c.bn == 64 && c.stages == 2)
    return launch_presplit_bn<64, 2>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, yh, yl, ldy, err, s);
  // persistent configurations: stages + 100
  if (c.bn == 128 && c.stages == 103)
    return launch_persistent_bn<128, 3>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, yh, yl, ldy, err, s);
  if (c.bn == 64 && c.stages == 104)
    return launch_persistent_bn<64, 4>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, yh, yl, ldy, err, s);
  return cudaErrorInvalidValue;
}

template <int BN, int NST>
cudaError_t launch_bn(int M, int N, int K, const float* x, int ldx, const float* W, const float* bias, int relu,
                      float* y, int ldy, int* err, cudaStream_t s) {
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(gemm_tf32x3_kernel<BN, NST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, Tf32Cfg<BN, NST>::SMEM);
      });
      e != cudaSuccess)
    return e;
  CUtensorMap ta, tb;
  if (!make_tmap_2d(&ta, 0, x, M, K, ldx, kBK, kBM) || !make_tmap_2d(&tb, 0, W, N, K, K, kBK, BN))
    return cudaErrorInvalidValue;
  dim3 grid(N / BN, (M + kBM - 1) / kBM);
  gemm_tf32x3_kernel<BN, NST><<<grid, 192, Tf32Cfg<BN, NST>::SMEM, s>>>(ta, tb, M, N, K, bias, relu, y, ldy, err);
  count_launch();
  return cudaGetLastError();
}

// (BN, stages): deep pipelines at 1 CTA per SM, shallow ones at 2 CTAs per SM.
const GemmCfg kTf32Cfgs[] = {{128, 3}, {64, 4}, {64, 2}};
// pre-split kernel: the above plus the persistent forms (stages + 100)
const GemmCfg kTf32PreCfgs[] = {{128, 3}, {64, 4}, {64, 2}, {128, 103}, {64, 104}};

cudaError_t launch_cfg(GemmCfg c, int M, int N, int K, const float* x, int ldx, const float* W, const float* bias,
                       int relu, float* y, int ldy, int* err, cudaStream_t s) {
  if (c.bn == 128 && c.stages == 3) return launch_bn<128, 3>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 64 && c.stages == 4) return launch_bn<64, 4>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 64 && c.stages == 2) return launch_bn<64, 2>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  return cudaErrorInvalidValue;
}

}  // namespace

void preload_tf32_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, gemm_tf32x3_presplit_kernel<128, 3>);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_presplit_kernel<64, 4>);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_presplit_kernel<64, 2>);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_persistent_kernel<128, 3>);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_persistent_kernel<64, 4>);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_persistent_head_kernel<128, 3>);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_persistent_head_kernel<64, 4>);
  cudaFuncGetAttributes(&fa, split_planes_kernel);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_kernel<128, 3>);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_kernel<64, 4>);
  cudaFuncGetAttributes(&fa, gemm_tf32x3_kernel<64, 2>);
}

int tf32_candidates(GemmCfg* out, int max) {
  int n = 0;
  for (const GemmCfg& c : kTf32Cfgs)
    if (n < max) out[n++] = c;
  return n;
}

int tf32_presplit_candidates(GemmCfg* out, int max) {
  int n = 0;
  for (const GemmCfg& c : kTf32PreCfgs)
    if (n < max) out[n++] = c;
  return n;
}

cudaError_t launch_linear_f32_tc(int M, int N, int K, const float* x, int ldx, const float* W, const float* bias,
                                 int relu, float* y, int ldy, int* err, cudaStream_t s, GemmCfg cfg) {
  if (M <= 0) return cudaSuccess;
  if (K <= 0 || (K % 4) || (N % 64) || (ldx % 4) || (ldy % 4) || (reinterpret_cast<uintptr_t>(x) & 15) ||
      (reinterpret_cast<uintptr_t>(W) & 15) || (reinterpret_cast<uintptr_t>(y) & 15))
    return cudaErrorInvalidValue;
  const int sms_n = device_sms();
  if (cfg.bn) {
    if (N % cfg.bn) return cudaErrorInvalidValue;
    return launch_cfg(cfg, M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  }
  const int mt = (M + kBM - 1) / kBM;
  if (N % 128 == 0 && mt * (N / 128) >= sms_n) return launch_bn<128, 3>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  return launch_bn<64, 4>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
}

cudaError_t launch_linear_f32_tc_presplit(int M, int N, int K, const float* xh, const float* xl, int ldx,
                                          const float* wh, const float* wl, const float* bias, int relu, float* yh,
                                          float* yl, int ldy, int* err, cudaStream_t s, GemmCfg cfg) {
  if (M <= 0) return cudaSuccess;
  if (K <= 0 || (K % 4) || (N % 64) || (ldx % 4) || (ldy % 4)) return cudaErrorInvalidValue;
  for (const void* p : {static_cast<const void*>(xh), static_cast<const void*>(xl), static_cast<const void*>(wh),
                        static_cast<const void*>(wl), static_cast<const void*>(yh), static_cast<const void*>(yl)})
    if (reinterpret_cast<uintptr_t>(p) & 15) return cudaErrorInvalidValue;
  const int sms_n = device_sms();
  if (cfg.bn) {
    if (N % cfg.bn) return cudaErrorInvalidValue;
    return launch_presplit_cfg(cfg, M, N, K, xh, xl, ldx, wh, wl, bias, relu, yh, yl, ldy, err, s);
  }
  const int mt = (M + kBM - 1) / kBM;
  if (N % 128 == 0 && mt * (N / 128) >= sms_n)
    return launch_presplit_bn<128, 3>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, yh, yl, ldy, err, s);
  return launch_presplit_bn<64, 4>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, yh, yl, ldy, err, s);
}

cudaError_t launch_linear_f32_tc_presplit_head(int M, int N, int K, const float* xh, const float* xl, int ldx,
                                               const float* wh, const float* wl, const float* bias, int relu,
                                               int* err, cudaStream_t s, GemmCfg cfg, const HeadParams& hp) {
  if (M <= 0) return cudaSuccess;
  if (!head_fusable(cfg, N) || K <= 0 || (K % 4) || (ldx % 4)) return cudaErrorInvalidValue;
  for (const void* p : {static_cast<const void*>(xh), static_cast<const void*>(xl), static_cast<const void*>(wh),
                        static_cast<const void*>(wl)})
    if (reinterpret_cast<uintptr_t>(p) & 15) return cudaErrorInvalidValue;
  if (cfg.bn == 128 && cfg.stages == 103)
    return launch_persistent_head_bn<128, 3>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, err, s, hp);
  if (cfg.bn == 64 && cfg.stages == 104)
    return launch_persistent_head_bn<64, 4>(M, N, K, xh, xl, ldx, wh, wl, bias, relu, err, s, hp);
  return cudaErrorInvalidValue;
}

cudaError_t launch_split_planes(const float* src, float* hi, float* lo, size_t n, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int blocks = static_cast<int>(std::min<size_t>((n + 255) / 256, 4096));
  split_planes_kernel<<<blocks, 256, 0, s>>>(src, hi, lo, n);
  count_launch();
  return cudaGetLastError();
}

}  // namespace sage
