// BF16 GEMM on the 5th-generation tensor cores (tcgen05) with TMA operand loads:
//     Y[M, N] = act(X[M, K] W[N, K]^T + b),  fp32 accumulation in tensor memory.
//
// One CTA computes a 128 x BN tile with 4 warps:
//   warp 0, one lane : TMA producer -- streams 128x64 tiles of X and BNx64 tiles of
//                      W (128-byte swizzle) into a STAGES-deep shared-memory ring;
//   warp 1, one lane : MMA issuer -- 4 tcgen05.mma (K = 16 each) per stage into a
//                      128 x BN fp32 accumulator in tensor memory; tcgen05.commit
//                      frees each stage and finally signals the epilogue;
//   all 4 warps      : epilogue -- tcgen05.ld of the warp's 32 TMEM lanes (= rows),
//                      bias, ReLU, round to bf16, 16-byte stores (possibly into a
//                      column slice of a wider buffer, e.g. the concat buffer).
// Every wait is bounded (see mbar_wait); a timed-out wait sets kErrTimeout in
// the caller's error word and the CTA finishes without hanging.  The K
// accumulation order of an output element is fixed (k-steps of 16 in order),
// so a row's result does not depend on M or on the other rows of the batch.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "kernels.h"

namespace sage {
namespace {

constexpr int kBM = 128, kBK = 64;

template <int BN, int NST>
struct TcCfg {
  static constexpr int A_BYTES = kBM * kBK * 2;
  static constexpr int B_BYTES = BN * kBK * 2;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int STAGES = NST;
  static constexpr int SMEM = STAGES * STAGE + 1024 + 256;
};

template <int BN, int NST>
__global__ void __launch_bounds__(128, 1)
    gemm_tc_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, int M, int N,
                   int K, const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ Y, int ldy,
                   int* err) {
  using C = TcCfg<BN, NST>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + C::STAGES * C::A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + C::STAGES * C::B_BYTES);
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
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (kb / C::STAGES) & 1;
      if (!mbar_wait(&empty[s], ph ^ 1, err)) break;
      mbar_arrive_expect_tx(&full[s], C::STAGE);
      tma_load_2d(sA + s * C::A_BYTES, &tmA, kb * kBK, m0, &full[s]);
      tma_load_2d(sB + s * C::B_BYTES, &tmB, kb * kBK, n0, &full[s]);
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    constexpr uint32_t idesc = idesc_bf16_f32(kBM, BN);
    for (int kb = 0; kb < KB; ++kb) {
      const int s = kb % C::STAGES;
      const uint32_t ph = (kb / C::STAGES) & 1;
      if (!mbar_wait(&full[s], ph, err)) break;
      tc_fence_after();
      const uint32_t a0 = smem_u32(sA + s * C::A_BYTES);
      const uint32_t b0 = smem_u32(sB + s * C::B_BYTES);
#pragma unroll
      for (int k = 0; k < kBK / 16; ++k) {
        tc_mma_bf16(tmem, sw128_kmajor_desc(a0 + k * 32), sw128_kmajor_desc(b0 + k * 32), idesc,
                    (kb | k) != 0 ? 1u : 0u);
      }
      tc_commit(&empty[s]);
    }
    tc_commit(accum);
  }
  __syncwarp();

  // ---- epilogue: TMEM -> registers -> bias/ReLU -> bf16 -> global
  mbar_wait(accum, 0, err);
  tc_fence_after();
  const int row = m0 + warp * 32 + lane;
  __nv_bfloat16* yrow = Y + static_cast<size_t>(row < M ? row : 0) * ldy + n0;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    uint32_t v[32];
    tmem_ld_32cols(tmem + (static_cast<uint32_t>(warp * 32) << 16) + c0, v);
    tmem_ld_wait();
    if (row < M) {
      uint32_t pk[16];
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        float f0 = __uint_as_float(v[2 * j]) + __ldg(bias + n0 + c0 + 2 * j);
        float f1 = __uint_as_float(v[2 * j + 1]) + __ldg(bias + n0 + c0 + 2 * j + 1);
        if (relu) {
          f0 = fmaxf(f0, 0.f);
          f1 = fmaxf(f1, 0.f);
        }
        pk[j] = pack_bf16x2(f0, f1);
      }
      uint4* dst = reinterpret_cast<uint4*>(yrow + c0);
#pragma unroll
      for (int q = 0; q < 4; ++q) dst[q] = make_uint4(pk[4 * q], pk[4 * q + 1], pk[4 * q + 2], pk[4 * q + 3]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, BN);
}

// Persistent form: one CTA per SM walks the output tiles (n fastest); two TMEM
// accumulators alternate so the epilogue of tile i overlaps the MMAs of tile i+1;
// the shared-memory ring runs on across tiles.  warp 0 lane 0: TMA; warp 1 lane 0:
// MMA; warps 2-5: epilogue (warp w reads TMEM lanes 32*(w%4)..+31).
// With HEAD the epilogue writes no Y: it fuses the sigmoid head (HeadParams) on
// the bf16-rounded activations, the values the separate head kernel would read.
// Without HEAD, a last wave of at most half as many tiles as CTAs runs as half-width
// items (B map tmB2 with boxes of BN / 2 rows), as in the fp32 persistent kernel.
template <int BN, int NST, bool HEAD>
__device__ __forceinline__ void tc_persistent_body(const CUtensorMap& tmA, const CUtensorMap& tmB, int M, int N,
                                                   int K, const float* __restrict__ bias, int relu,
                                                   __nv_bfloat16* __restrict__ Y, int ldy, int* err,
                                                   const HeadParams* hp, const CUtensorMap* tmB2 = nullptr) {
  using C = TcCfg<BN, NST>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + C::STAGES * C::A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + C::STAGES * C::B_BYTES);
  uint64_t* empty = full + C::STAGES;
  uint64_t* acc_full = empty + C::STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int KB = (K + kBK - 1) / kBK;
  const int NT = N / BN, MT = (M + kBM - 1) / kBM;
  const int tiles = NT * MT;
  const int GR = static_cast<int>(gridDim.x);
  int nfull = tiles, items = tiles;
  if (!HEAD && tmB2 && tiles > GR && tiles % GR != 0 && 2 * (tiles % GR) <= GR) {
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
    tma_prefetch_desc(&tmA);
    tma_prefetch_desc(&tmB);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
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
          mbar_arrive_expect_tx(&full[s], whole ? C::STAGE : C::STAGE - C::B_BYTES / 2);
          tma_load_2d(sA + s * C::A_BYTES, &tmA, kb * kBK, m0, &full[s]);
          tma_load_2d(sB + s * C::B_BYTES, whole ? &tmB : tmB2, kb * kBK, n0, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc_whole = idesc_bf16_f32(kBM, BN), idesc_half = idesc_bf16_f32(kBM, BN / 2);
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
          const uint32_t a0 = smem_u32(sA + s * C::A_BYTES);
          const uint32_t b0 = smem_u32(sB + s * C::B_BYTES);
#pragma unroll
          for (int k = 0; k < kBK / 16; ++k)
            tc_mma_bf16(acc, sw128_kmajor_desc(a0 + k * 32), sw128_kmajor_desc(b0 + k * 32), idesc,
                        (kb | k) != 0 ? 1u : 0u);
          tc_commit(&empty[s]);
        }
        tc_commit(&acc_full[buf]);
      }
    }
  } else {
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
        const unsigned G = static_cast<unsigned>(N / 64);
        const __nv_bfloat16* hw = static_cast<const __nv_bfloat16*>(hp->f.w) + n0;
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
              const float ob = __bfloat162float(__float2bfloat16_rn(o));
              p[j] = __fmul_rn(ob, __bfloat162float(hw[c0 + 32 * half + j]));
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
      __nv_bfloat16* yrow = Y + static_cast<size_t>(row < M ? row : 0) * ldy + n0;
#pragma unroll 1
      for (int c0 = 0; c0 < width; c0 += 32) {
        uint32_t v[32];
        tmem_ld_32cols(tmem + static_cast<uint32_t>(buf * BN) + (static_cast<uint32_t>(q * 32) << 16) + c0, v);
        tmem_ld_wait();
        if (row < M) {
          uint32_t pk[16];
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            float f0 = __uint_as_float(v[2 * j]) + __ldg(bias + n0 + c0 + 2 * j);
            float f1 = __uint_as_float(v[2 * j + 1]) + __ldg(bias + n0 + c0 + 2 * j + 1);
            if (relu) {
              f0 = fmaxf(f0, 0.f);
              f1 = fmaxf(f1, 0.f);
            }
            pk[j] = pack_bf16x2(f0, f1);
          }
          uint4* dst = reinterpret_cast<uint4*>(yrow + c0);
#pragma unroll
          for (int u = 0; u < 4; ++u) dst[u] = make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
        }
      }
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
    gemm_tc_persistent_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                              const __grid_constant__ CUtensorMap tmB2, int M, int N, int K,
                              const float* __restrict__ bias, int relu, __nv_bfloat16* __restrict__ Y, int ldy,
                              int* err) {
  tc_persistent_body<BN, NST, false>(tmA, tmB, M, N, K, bias, relu, Y, ldy, err, nullptr, &tmB2);
}

template <int BN, int NST>
__global__ void __launch_bounds__(192, 1)
    gemm_tc_persistent_head_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                                   int M, int N, int K, const float* __restrict__ bias, int relu, int* err,
                                   const __grid_constant__ HeadParams hp) {
  tc_persistent_body<BN, NST, true>(tmA, tmB, M, N, K, bias, relu, nullptr, 0, err, &hp);
}

// Row-major bf16 matrix [rows, cols] with row stride ld elements, tiles of
// box_rows x 64 columns, 128-byte swizzle, zero fill outside the matrix.
bool make_map(CUtensorMap* m, const void* base, int rows, int cols, int ld, int box_rows) {
  return make_tmap_2d(m, 1, base, rows, cols, ld, kBK, box_rows);
}

template <int BN, int NST>
cudaError_t launch_bn(int M, int N, int K, const void* x, int ldx, const void* W, const float* bias, int relu,
                      void* y, int ldy, int* err, cudaStream_t s) {
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(gemm_tc_kernel<BN, NST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN, NST>::SMEM);
      });
      e != cudaSuccess)
    return e;
  CUtensorMap ta, tb;
  if (!make_map(&ta, x, M, K, ldx, kBM) || !make_map(&tb, W, N, K, K, BN)) return cudaErrorInvalidValue;
  dim3 grid(N / BN, (M + kBM - 1) / kBM);
  gemm_tc_kernel<BN, NST><<<grid, 128, TcCfg<BN, NST>::SMEM, s>>>(ta, tb, M, N, K, bias, relu,
                                                                static_cast<__nv_bfloat16*>(y), ldy, err);
  count_launch();
  return cudaGetLastError();
}

template <int BN, int NST>
cudaError_t launch_persistent_bn(int M, int N, int K, const void* x, int ldx, const void* W, const float* bias,
                                 int relu, void* y, int ldy, int* err, cudaStream_t s) {
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(gemm_tc_persistent_kernel<BN, NST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN, NST>::SMEM);
      });
      e != cudaSuccess)
    return e;
  CUtensorMap ta, tb, tb2;
  if (!make_map(&ta, x, M, K, ldx, kBM) || !make_map(&tb, W, N, K, K, BN) || !make_map(&tb2, W, N, K, K, BN / 2))
    return cudaErrorInvalidValue;
  const int tiles = (N / BN) * ((M + kBM - 1) / kBM);
  const int sms_n = device_sms();
  const int grid = tiles < sms_n ? tiles : sms_n;
  gemm_tc_persistent_kernel<BN, NST><<<grid, 192, TcCfg<BN, NST>::SMEM, s>>>(
      ta, tb, tb2, M, N, K, bias, relu, static_cast<__nv_bfloat16*>(y), ldy, err);
  count_launch();
  return cudaGetLastError();
}

template <int BN, int NST>
cudaError_t launch_persistent_head_bn(int M, int N, int K, const void* x, int ldx, const void* W, const float* bias,
                                      int relu, int* err, cudaStream_t s, const HeadParams& hp) {
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(gemm_tc_persistent_head_kernel<BN, NST>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, TcCfg<BN, NST>::SMEM);
      });
      e != cudaSuccess)
    return e;
  CUtensorMap ta, tb;
  if (!make_map(&ta, x, M, K, ldx, kBM) || !make_map(&tb, W, N, K, K, BN)) return cudaErrorInvalidValue;
  const int tiles = (N / BN) * ((M + kBM - 1) / kBM);
  const int sms_n = device_sms();
  const int grid = tiles < sms_n ? tiles : sms_n;
  gemm_tc_persistent_head_kernel<BN, NST><<<grid, 192, TcCfg<BN, NST>::SMEM, s>>>(ta, tb, M, N, K, bias, relu, err,
                                                                                  hp);
  count_launch();
  return cudaGetLastError();
}

// Tile shapes the bf16 GEMM can run: (BN, stages).  The deep pipelines use
// 192 KB of shared memory (one CTA per SM); the shallow ones ~100 KB (two CTAs
// per SM, so one CTA's epilogue overlaps the other's main loop).
const GemmCfg kBf16Cfgs[] = {{256, 4}, {128, 6}, {64, 8}, {256, 2}, {128, 3}, {64, 4},
                              {256, 104}, {128, 106}};  // stages >= 100: persistent

cudaError_t launch_cfg(GemmCfg c, int M, int N, int K, const void* x, int ldx, const void* W, const float* bias,
                       int relu, void* y, int ldy, int* err, cudaStream_t s) {
  if (c.bn == 256 && c.stages == 4) return launch_bn<256, 4>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 128 && c.stages == 6) return launch_bn<128, 6>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 64 && c.stages == 8) return launch_bn<64, 8>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 256 && c.stages == 2) return launch_bn<256, 2>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 128 && c.stages == 3) return launch_bn<128, 3>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 64 && c.stages == 4) return launch_bn<64, 4>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 256 && c.stages == 104)
    return launch_persistent_bn<256, 4>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (c.bn == 128 && c.stages == 106)
    return launch_persistent_bn<128, 6>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  return cudaErrorInvalidValue;
}

}  // namespace

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    cudaDriverEntryPointQueryResult q;
    void* p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

bool make_tmap_2d(CUtensorMap* m, int dtype, const void* base, int rows, int cols, int ld, int box_cols,
                  int box_rows) {
  auto enc = encode_fn();
  if (!enc) return false;
  const int es = dtype == 1 ? 2 : 4;
  cuuint64_t dims[2] = {static_cast<cuuint64_t>(cols), static_cast<cuuint64_t>(rows)};
  cuuint64_t strides[1] = {static_cast<cuuint64_t>(ld) * es};
  cuuint32_t box[2] = {static_cast<cuuint32_t>(box_cols), static_cast<cuuint32_t>(box_rows)};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = enc(m, dtype == 1 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                   const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                   CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

void preload_tc_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, gemm_tc_kernel<256, 4>);
  cudaFuncGetAttributes(&fa, gemm_tc_kernel<128, 6>);
  cudaFuncGetAttributes(&fa, gemm_tc_kernel<64, 8>);
  cudaFuncGetAttributes(&fa, gemm_tc_kernel<256, 2>);
  cudaFuncGetAttributes(&fa, gemm_tc_kernel<128, 3>);
  cudaFuncGetAttributes(&fa, gemm_tc_kernel<64, 4>);
  cudaFuncGetAttributes(&fa, gemm_tc_persistent_kernel<256, 4>);
  cudaFuncGetAttributes(&fa, gemm_tc_persistent_kernel<128, 6>);
  cudaFuncGetAttributes(&fa, gemm_tc_persistent_head_kernel<256, 4>);
  cudaFuncGetAttributes(&fa, gemm_tc_persistent_head_kernel<128, 6>);
  encode_fn();
}

int gemm_candidates(int kind, GemmCfg* out, int max) {
  int n = 0;
  if (kind == kGemmBf16) {
    for (const GemmCfg& c : kBf16Cfgs)
      if (n < max) out[n++] = c;
  } else if (kind == kGemmTf32Pre) {
    n = tf32_presplit_candidates(out, max);
  } else if (kind == kBottom01) {
    n = bottom01_candidates(out, max);
  } else if (kind == kGatherTop0) {
    // the gather and the first top layer in one kernel, or separate kernels
    const GemmCfg c[2] = {{256, 2}, {1, 1}};
    for (const GemmCfg& x : c)
      if (n < max) out[n++] = x;
  } else {
    n = tf32_candidates(out, max);
  }
  return n;
}

cudaError_t launch_linear_bf16_tc(int M, int N, int K, const void* x, int ldx, const void* W,
                                  const float* bias, int relu, void* y, int ldy, int* err, cudaStream_t s,
                                  GemmCfg cfg) {
  if (M <= 0) return cudaSuccess;
  if (K <= 0 || (K % kBK) || (N % 64) || (ldx % 8) || (ldy % 8) ||
      (reinterpret_cast<uintptr_t>(x) & 15) || (reinterpret_cast<uintptr_t>(W) & 15) ||
      (reinterpret_cast<uintptr_t>(y) & 15))
    return cudaErrorInvalidValue;
  const int sms_n = device_sms();
  if (cfg.bn) {
    if (N % cfg.bn) return cudaErrorInvalidValue;
    return launch_cfg(cfg, M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  }
  const int mt = (M + kBM - 1) / kBM;
  if (N % 256 == 0 && mt * (N / 256) >= sms_n) return launch_bn<256, 4>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  if (N % 128 == 0 && mt * (N / 128) >= sms_n) return launch_bn<128, 6>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
  return launch_bn<64, 8>(M, N, K, x, ldx, W, bias, relu, y, ldy, err, s);
}

cudaError_t launch_linear_bf16_tc_head(int M, int N, int K, const void* x, int ldx, const void* W,
                                       const float* bias, int relu, int* err, cudaStream_t s, GemmCfg cfg,
                                       const HeadParams& hp) {
  if (M <= 0) return cudaSuccess;
  if (!head_fusable(cfg, N) || K <= 0 || (K % kBK) || (ldx % 8) || (reinterpret_cast<uintptr_t>(x) & 15) ||
      (reinterpret_cast<uintptr_t>(W) & 15))
    return cudaErrorInvalidValue;
  if (cfg.bn == 256 && cfg.stages == 104)
    return launch_persistent_head_bn<256, 4>(M, N, K, x, ldx, W, bias, relu, err, s, hp);
  if (cfg.bn == 128 && cfg.stages == 106)
    return launch_persistent_head_bn<128, 6>(M, N, K, x, ldx, W, bias, relu, err, s, hp);
  return cudaErrorInvalidValue;
}

}  // namespace sage
