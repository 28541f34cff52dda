// The gather and the first top layer of an fp32 function in one persistent kernel.
//
// Unfused, the gather writes every pooled bag of the batch into the concat buffer
// (as tf32 hi / fp32 residual lo planes, 8 bytes per element) and the first top
// layer's tensor-core GEMM reads it back with the TMA.  Here the GEMM's own
// producer warps gather a table's bags for the tile's 128 rows and write the sums
// straight into the shared-memory A tiles, in the 128-byte-swizzle layout the TMA
// would have produced; the pooled columns never reach memory.  The bottom MLP's
// output (the concat buffer's last columns, written by the bottom kernels before
// this one starts) still comes in through the TMA as the last k-blocks.
//
// One CTA owns a whole 128-row tile across all N0 (256 or 512) output columns, so
// no row is gathered twice: its fp32 accumulator takes N0 of the 512 TMEM columns,
// and each 32-column k-block runs as N0 / 256 MMAs of 128 x 256 per product.
//   warp 0 lane 0 : TMA -- the weight planes (B) per (k-block, 256-column half) into
//                   a two-slot ring, the bottom output's A tiles
//   warp 1 lane 0 : MMA issuer, three tf32 products per k-step (hi.hi, hi.lo, lo.hi)
//   warps 2-5     : epilogue, bias + ReLU, output as hi/lo planes
//   warps 6..     : producers, P warps of four 8-lane groups; group g sums the bags
//                   of rows g, g + 4P, ... of the tile, lane l the columns
//                   [8l, 8l + 8) of the table's 64 (two 16-byte pieces of a row)
// A table's 64 columns are two k-blocks, so the A ring has two stages: while the
// tensor cores work on table t, the producers already gather table t + 1 into
// registers and wait only to store it.
//
// The sums are those of the lane-group gather kernel -- each lane adds its pieces of
// a bag's rows in bag order, fp32, from zero -- and the hi/lo split and the MMA
// sequence over the k-blocks are those of the unfused path, so the first top
// layer's output is bitwise the unfused chain's.
#include "kernels.h"

namespace sage {
namespace {

constexpr int kBM = 128, kBK = 32, kBH = 256;  // tile rows, k-block columns, MMA N (a half)

template <int NH>
struct GTCfg {
  static constexpr int A_BYTES = kBM * kBK * 4;       // one plane of one k-block: 16 KB
  static constexpr int A_STAGE = 2 * A_BYTES;         // hi + lo
  static constexpr int B_BYTES = kBH * kBK * 4;       // one plane of one (k-block, half): 32 KB
  static constexpr int B_SLOT = 2 * B_BYTES;
  static constexpr int SMEM = 2 * A_STAGE + 2 * B_SLOT + 1024 + 256;
  static_assert(SMEM <= 232448, "shared memory");
};

__device__ __forceinline__ uint4 ldg_nc(const uint4* p) { return __ldg(p); }

// acc += one 16-byte piece of a row: four round-to-nearest fp32 additions, as two
// paired adds (the gather kernel's instruction and order).
__device__ __forceinline__ void add4(float* acc, const uint4& v) {
  asm("{\n\t.reg .b64 a, b;\n\tmov.b64 a, {%0, %1};\n\tmov.b64 b, {%4, %5};\n\t"
      "add.rn.f32x2 a, a, b;\n\tmov.b64 {%0, %1}, a;\n\t"
      "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%6, %7};\n\tadd.rn.f32x2 a, a, b;\n\tmov.b64 {%2, %3}, a;\n\t}"
      : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
      : "f"(__uint_as_float(v.x)), "f"(__uint_as_float(v.y)), "f"(__uint_as_float(v.z)), "f"(__uint_as_float(v.w)));
}

template <int NH, int P, int U>
__global__ void __launch_bounds__(192 + 32 * P, 1)
    gather_top0_kernel(const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                       const __grid_constant__ CUtensorMap tmXh, const __grid_constant__ CUtensorMap tmXl,
                       const __grid_constant__ GatherArgs ga, const __grid_constant__ InvTable tab, int K0,
                       const float* __restrict__ b0, float* __restrict__ Yh, float* __restrict__ Yl, int ldy,
                       int* err) {
  using C = GTCfg<NH>;
  constexpr int NP = 32 * P;  // producer threads
  constexpr int N0 = NH * kBH;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_align1024(smem_raw);
  auto a_hi = [&](int s) { return smem + s * C::A_STAGE; };
  auto a_lo = [&](int s) { return smem + s * C::A_STAGE + C::A_BYTES; };
  auto b_hi = [&](int s) { return smem + 2 * C::A_STAGE + s * C::B_SLOT; };
  auto b_lo = [&](int s) { return smem + 2 * C::A_STAGE + s * C::B_SLOT + C::B_BYTES; };
  uint64_t* afull = reinterpret_cast<uint64_t*>(smem + 2 * C::A_STAGE + 2 * C::B_SLOT);
  uint64_t* aempty = afull + 2;
  uint64_t* bfull = aempty + 2;
  uint64_t* bempty = bfull + 2;
  uint64_t* acc_full = bempty + 2;
  uint64_t* acc_empty = acc_full + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = tab.M, T = ga.T;
  const int KB = K0 / kBK, KG = 2 * T;  // k-blocks in all; those the producers gather
  const int tiles = (M + kBM - 1) / kBM;

  if (warp == 0) tmem_alloc(tmem_slot, N0);
  if (warp == 1 && lane == 0) {
    for (int s = 0; s < 2; ++s) {
      mbar_init(&afull[s], 1 + NP);  // the TMA thread + every producer thread, every k-block
      mbar_init(&aempty[s], 1);
      mbar_init(&bfull[s], 1);
      mbar_init(&bempty[s], 1);
    }
    mbar_init(acc_full, 1);
    mbar_init(acc_empty, 128);
    fence_mbar_init();
  }
  if (warp == 2 && lane == 0) {
    tma_prefetch_desc(&tmBh);
    tma_prefetch_desc(&tmBl);
    tma_prefetch_desc(&tmXh);
    tma_prefetch_desc(&tmXl);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t gk = 0, gb = 0;  // k-block and B-slot use counters across tiles
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int m0 = t * kBM;
        for (int kb = 0; kb < KB && ok; ++kb, ++gk) {
          const int s = gk & 1;
          if (!mbar_wait(&aempty[s], ((gk >> 1) & 1) ^ 1, err)) {
            ok = false;
            break;
          }
          if (kb >= KG) {
            // the bottom MLP's output: concat columns [kb * 32, kb * 32 + 32)
            mbar_arrive_expect_tx(&afull[s], C::A_STAGE);
            tma_load_2d(a_hi(s), &tmXh, kb * kBK, m0, &afull[s]);
            tma_load_2d(a_lo(s), &tmXl, kb * kBK, m0, &afull[s]);
          } else {
            mbar_arrive(&afull[s]);
          }
          for (int h = 0; h < NH; ++h, ++gb) {
            const int sb = gb & 1;
            if (!mbar_wait(&bempty[sb], ((gb >> 1) & 1) ^ 1, err)) {
              ok = false;
              break;
            }
            mbar_arrive_expect_tx(&bfull[sb], C::B_SLOT);
            tma_load_2d(b_hi(sb), &tmBh, kb * kBK, h * kBH, &bfull[sb]);
            tma_load_2d(b_lo(sb), &tmBl, kb * kBK, h * kBH, &bfull[sb]);
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32_f32(kBM, kBH);
      uint32_t gk = 0, gb = 0;
      int i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++i) {
        if (!mbar_wait(acc_empty, (i & 1) ^ 1, err)) break;
        tc_fence_after();
        for (int kb = 0; kb < KB && ok; ++kb, ++gk) {
          const int s = gk & 1;
          if (!mbar_wait(&afull[s], (gk >> 1) & 1, err)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t ah = smem_u32(a_hi(s)), al = smem_u32(a_lo(s));
          for (int h = 0; h < NH; ++h, ++gb) {
            const int sb = gb & 1;
            if (!mbar_wait(&bfull[sb], (gb >> 1) & 1, err)) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t acc = tmem + static_cast<uint32_t>(h * kBH);
            const uint32_t bh = smem_u32(b_hi(sb)), bl = smem_u32(b_lo(sb));
#pragma unroll
            for (int k = 0; k < kBK / 8; ++k) {
              const uint32_t o = k * 32;
              tc_mma_tf32_fill_a(acc, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bh + o), idesc,
                                 (kb | k) != 0 ? 1u : 0u);
              tc_mma_tf32_lastuse_a(acc, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bl + o), idesc, 1u);
              tc_mma_tf32(acc, sw128_kmajor_desc(al + o), sw128_kmajor_desc(bh + o), idesc, 1u);
            }
            tc_commit(&bempty[sb]);
          }
          tc_commit(&aempty[s]);
        }
        if (ok) tc_commit(acc_full);
      }
    }
  } else if (warp < 6) {
    // ---- epilogue: row m0 + 32q + lane, every column; bias, ReLU, hi/lo planes
    const int q = warp & 3;
    int i = 0;
    for (int t = blockIdx.x; t < tiles; t += gridDim.x, ++i) {
      if (!mbar_wait(acc_full, i & 1, err)) break;
      tc_fence_after();
      const int row = t * kBM + q * 32 + lane;
      const size_t ro = static_cast<size_t>(row < M ? row : 0) * ldy;
#pragma unroll 1
      for (int c0 = 0; c0 < N0; c0 += 32) {
        uint32_t v[32];
        tmem_ld_32cols(tmem + (static_cast<uint32_t>(q * 32) << 16) + c0, v);
        tmem_ld_wait();
        if (row < M) {
          float4* dh = reinterpret_cast<float4*>(Yh + ro + c0);
          float4* dl = reinterpret_cast<float4*>(Yl + ro + c0);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) o[u] = fmaxf(__uint_as_float(v[4 * j + u]) + __ldg(b0 + c0 + 4 * j + u), 0.f);
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
      mbar_arrive(acc_empty);
    }
  } else {
    // ---- producers
    constexpr int NGRP = 4 * P;  // lane groups; each takes rows grp, grp + NGRP, ... of a tile
    static_assert(kBM % NGRP == 0, "every lane group of a warp takes the same number of rows");
    const int grp = (warp - 6) * 4 + (lane >> 3);
    const int gl = lane & 7;
    const int half = gl >> 2;             // k-block of the table's two that lane gl's columns fall in
    const uint32_t c0 = (gl & 3) * 2;     // its two 16-byte chunks in that k-block's 128-byte row
    uint32_t gk = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      const int m0 = t * kBM;
      for (int tb = 0; tb < T && ok; ++tb) {
        // this table's k-blocks 2tb, 2tb + 1 use A stages gk & 1 and (gk + 1) & 1
        const uint32_t g0 = gk + 2 * tb;
        const int sm = static_cast<int>((g0 + half) & 1);
        const char* tbase = ga.tables + ga.table_off[tb] + gl * 32;
        const unsigned rows = static_cast<unsigned>(ga.table_rows[tb]);
        bool waited = false;
        for (int r = grp; r < kBM; r += NGRP) {
          const int row = m0 + r;
          int64_t beg = 0, end = 0;
          const int32_t* idx = nullptr;
          if (row < M) {
            const int inv = tab.n == 1 ? 0 : find_inv(tab, row);
            const InvDesc& d = tab.d[inv];
            const int64_t bag = static_cast<int64_t>(tb) * d.batch + (row - d.row_base);
            beg = d.offsets[bag];
            end = d.offsets[bag + 1];
            idx = d.indices + beg;
          }
          const int len = static_cast<int>(end - beg);
          int maxlen = len;
#pragma unroll
          for (int o = 8; o < 32; o <<= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
          float acc[2][4];
#pragma unroll
          for (int w = 0; w < 2; ++w)
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[w][e] = 0.f;
          // the group's next 32 indices, four loads per lane: position j0 + 8m + gl in register m
          for (int j0 = 0; j0 < maxlen; j0 += 32) {
            int my[4];
#pragma unroll
            for (int m = 0; m < 4; ++m) my[m] = j0 + m * 8 + gl < len ? __ldg(idx + j0 + m * 8 + gl) : 0;
            const int cnt = min(32, maxlen - j0);
            for (int p = 0; p < cnt; p += U) {
              uint4 v[U][2];
              bool okr[U];
              const int mp = p >> 3;
              int src = my[0];
#pragma unroll
              for (int m = 1; m < 4; ++m) src = mp == m ? my[m] : src;
#pragma unroll
              for (int u = 0; u < U; ++u) {
                const int qq = p + u;
                const int rw = __shfl_sync(0xffffffffu, src, (lane & ~7) + (qq & 7));
                okr[u] = qq < cnt && j0 + qq < len;
                if (okr[u] && static_cast<unsigned>(rw) >= rows) {
                  okr[u] = false;
                  if (err) atomicOr(err, kErrBounds);
                }
                const uint4* sp = reinterpret_cast<const uint4*>(tbase + static_cast<size_t>(okr[u] ? rw : 0) * 256);
                v[u][0] = okr[u] ? ldg_nc(sp) : make_uint4(0, 0, 0, 0);
                v[u][1] = okr[u] ? ldg_nc(sp + 1) : make_uint4(0, 0, 0, 0);
              }
#pragma unroll
              for (int u = 0; u < U; ++u) {
                if (!okr[u]) continue;
                add4(acc[0], v[u][0]);
                add4(acc[1], v[u][1]);
              }
            }
          }
          if (!waited) {
            // both of the table's stages must be free before the first store
            waited = true;
            if (!mbar_wait(&aempty[g0 & 1], ((g0 >> 1) & 1) ^ 1, err) ||
                !mbar_wait(&aempty[(g0 + 1) & 1], (((g0 + 1) >> 1) & 1) ^ 1, err)) {
              ok = false;
            }
          }
          if (ok) {
            // row r of the A tile: chunk c of its 128-byte row at slot c ^ (r % 8)
            const uint32_t rb = static_cast<uint32_t>((r >> 3) * 1024 + (r & 7) * 128);
#pragma unroll
            for (int w = 0; w < 2; ++w) {
              float hh[4], ll[4];
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                hh[e] = to_tf32_rna(acc[w][e]);
                ll[e] = acc[w][e] - hh[e];
              }
              const uint32_t off = rb + (((c0 + w) ^ static_cast<uint32_t>(r & 7)) << 4);
              *reinterpret_cast<float4*>(a_hi(sm) + off) = make_float4(hh[0], hh[1], hh[2], hh[3]);
              *reinterpret_cast<float4*>(a_lo(sm) + off) = make_float4(ll[0], ll[1], ll[2], ll[3]);
            }
          }
        }
        if (!ok) break;
        fence_proxy_async_smem();  // generic-proxy stores -> the tensor cores' reads
        mbar_arrive(&afull[g0 & 1]);
        mbar_arrive(&afull[(g0 + 1) & 1]);
      }
      // the bottom output's k-blocks come by TMA: only keep the stage phases in step
      for (int kb = KG; kb < KB && ok; ++kb) {
        const uint32_t g = gk + kb;
        if (!mbar_wait(&aempty[g & 1], ((g >> 1) & 1) ^ 1, err)) {
          ok = false;
          break;
        }
        mbar_arrive(&afull[g & 1]);
      }
      gk += KB;
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, N0);
}

constexpr int kP = 16, kU = 4;

template <int NH>
cudaError_t launch_nh(const GatherArgs& a, const InvTable& tab, int K0, const CUtensorMap& tbh, const CUtensorMap& tbl,
                      const CUtensorMap& txh, const CUtensorMap& txl, const float* b0, float* yh, float* yl, int ldy,
                      int* err, cudaStream_t s) {
  using C = GTCfg<NH>;
  auto kern = gather_top0_kernel<NH, kP, kU>;
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(gather_top0_kernel<NH, kP, kU>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    C::SMEM);
      });
      e != cudaSuccess)
    return e;
  const int tiles = (tab.M + kBM - 1) / kBM;
  const int sms = device_sms();
  const int grid = tiles < sms ? tiles : sms;
  kern<<<grid, 192 + 32 * kP, C::SMEM, s>>>(tbh, tbl, txh, txl, a, tab, K0, b0, yh, yl, ldy, err);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

bool gather_top0_fusable(int dtype, int dim, int T, int n_bot_out, int N0, bool presplit) {
  return dtype == 0 && presplit && dim == 64 && T >= 1 && n_bot_out > 0 && n_bot_out % kBK == 0 &&
         (N0 == 256 || N0 == 512);
}

cudaError_t launch_gather_top0_f32(const GatherArgs& a, const InvTable& tab, int N0, int K0, const float* xh,
                                   const float* xl, int ldx, const float* wh, const float* wl, const float* b0,
                                   float* yh, float* yl, int ldy, int* err, cudaStream_t s) {
  if (tab.M <= 0) return cudaSuccess;
  const int nbot = K0 - a.T * 64;  // the bottom output's columns, after the T tables' 64 each
  if (a.dtype != 0 || a.dim != 64 || a.T < 1 || a.T > kMaxTables || tab.n < 1 || tab.n > kMaxInv || nbot <= 0 ||
      (nbot % kBK) || (N0 != 256 && N0 != 512) || (ldx % 4) || (ldy % 4) || K0 > ldx || ldy < N0)
    return cudaErrorInvalidValue;
  CUtensorMap tbh, tbl, txh, txl;
  if (!make_tmap_2d(&tbh, 0, wh, N0, K0, K0, kBK, kBH) || !make_tmap_2d(&tbl, 0, wl, N0, K0, K0, kBK, kBH) ||
      !make_tmap_2d(&txh, 0, xh, tab.M, K0, ldx, kBK, kBM) || !make_tmap_2d(&txl, 0, xl, tab.M, K0, ldx, kBK, kBM))
    return cudaErrorInvalidValue;
  return N0 == 512 ? launch_nh<2>(a, tab, K0, tbh, tbl, txh, txl, b0, yh, yl, ldy, err, s)
                   : launch_nh<1>(a, tab, K0, tbh, tbl, txh, txl, b0, yh, yl, ldy, err, s);
}

void preload_gather_top0_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, gather_top0_kernel<1, kP, kU>);
  cudaFuncGetAttributes(&fa, gather_top0_kernel<2, kP, kU>);
}

}  // namespace sage
