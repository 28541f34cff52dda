// Bottom layers 0 and 1 (and optionally 2) of an fp32 function in one persistent
// kernel.
//
// Layer 0 (K0 <= 15 dense inputs -> N0 outputs, ReLU) has too little arithmetic for
// the tensor cores and would otherwise write N0 activations per row (as two tf32
// planes) only for layer 1 to read them back.  Here sixteen producer warps compute
// each 128 x 32 k-block of layer 0's output straight into the shared-memory A
// tiles of layer 1 -- tf32 hi / fp32 residual lo, in the 128-byte-swizzle layout
// the TMA would have written -- while layer 1 runs on the tensor cores as three
// tf32 products (hi.hi + hi.lo + lo.hi), exactly as the persistent kernel does:
//   warp 0 lane 0 : TMA of layer 1's weight planes (B)
//   warp 1 lane 0 : MMA issuer, two TMEM accumulators alternating between tiles
//   warps 2-5     : epilogue (bias, ReLU, hi/lo planes of layer 1's output; a CTA's
//                   last tile leaves through the idle stage ring and TMA stores)
//   warps 6-21    : producers, thread = row of the tile, four warps per row set
//                   (each computing a quarter of a k-block's 32 columns)
// Layer 0's arithmetic is bottom0's (fmaf chain over k = 0..15 with zero padding,
// then + bias, ReLU), so the fused and separate forms give the same bits.  The bias
// sits in weight slot K0 against an input of 1: fmaf(1, b, s) rounds s + b once, as
// the separate kernel's addition does, and the zero-padded terms after it leave the
// sum unchanged (an fmaf chain from +0 reaches -0 only by underflow), so no global
// load remains in the producers' loop.
#include "kernels.h"

namespace sage {
namespace {

constexpr int kBM = 128, kBK = 32, kKM = 16, kW0Max = 512;
// producer warps: kGroups sets of 4, set g computing chunks [g * 8 / kGroups, ...) of
// each k-block's 8 16-byte column chunks for its 128 rows
constexpr int kGroups = 4, kProducers = 128 * kGroups, kThreads = 192 + kProducers;

template <int BN, int NST>
struct B01Cfg {
  static constexpr int A_BYTES = kBM * kBK * 4;
  static constexpr int B_BYTES = BN * kBK * 4;
  static constexpr int STAGE = 2 * (A_BYTES + B_BYTES);
  static constexpr int W0_BYTES = kW0Max * kKM * 4;  // layer 0's weights, rows padded to 16
  static constexpr int SMEM = NST * STAGE + W0_BYTES + 1024 + 512;
  static_assert(SMEM <= 232448, "shared memory");
  static_assert(NST * STAGE >= 20 * 8192, "last-tile output staging: 8 KB per epilogue and producer warp");
};

// Layer 2 of the bottom MLP, when the kernel also computes it (N2 outputs from
// layer 1's BN = N1 outputs): its weight planes and bias.
struct Layer2 {
  CUtensorMap wh, wl;  // W2 hi / lo planes, [N2, N1]
  const float* b;      // [N2]
  int n;               // N2
};

// L2: the kernel also computes layer 2.  Every CTA then owns one tile whose rows are
// complete (BN = N1), so after layer 1's MMAs the whole stage ring is free for
// layer 2: rounds of up to h k-blocks, each a 128 x 32 block of ReLU(acc1 + b1)
// written as hi/lo A tiles by the 20 worker warps (epilogue and producer warps)
// and the matching W2 planes loaded by TMA, three tf32 MMAs per k-step into a
// second accumulator (TMEM columns BN..BN+N2).  Layer 1's output is never stored;
// `tmYh` / `tmYl` then describe layer 2's output.
template <int BN, int NST, bool L2>
__global__ void __launch_bounds__(kThreads, 1)
    bottom01_kernel(const __grid_constant__ CUtensorMap tmBh, const __grid_constant__ CUtensorMap tmBl,
                    const __grid_constant__ CUtensorMap tmYh, const __grid_constant__ CUtensorMap tmYl,
                    const __grid_constant__ InvTable tab, int K0, int N0, const float* __restrict__ W0,
                    const float* __restrict__ b0, int N1, const float* __restrict__ b1, float* __restrict__ Yh,
                    float* __restrict__ Yl, int ldy, int* err, const __grid_constant__ Layer2 l2) {
  using C = B01Cfg<BN, NST>;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = smem_align1024(smem_raw);
  auto a_hi = [&](int s) { return smem + s * C::STAGE; };
  auto b_hi = [&](int s) { return smem + s * C::STAGE + C::A_BYTES; };
  auto a_lo = [&](int s) { return smem + s * C::STAGE + C::A_BYTES + C::B_BYTES; };
  auto b_lo = [&](int s) { return smem + s * C::STAGE + 2 * C::A_BYTES + C::B_BYTES; };
  float* sW0 = reinterpret_cast<float*>(smem + NST * C::STAGE);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + NST * C::STAGE + C::W0_BYTES);
  uint64_t* empty = full + NST;
  uint64_t* acc_full = empty + NST;  // [2]
  uint64_t* acc_empty = acc_full + 2;  // [2]
  uint64_t* w2full = acc_empty + 2;    // layer 2: W2 planes of a round loaded
  uint64_t* a2full = w2full + 1;       // layer 2: A tiles of a round written
  uint64_t* l2done = a2full + 1;       // layer 2: a round's MMAs complete
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(l2done + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int M = tab.M;
  const int KB = N0 / kBK;  // layer 1's reduction runs over layer 0's outputs
  const int NT = N1 / BN, MT = (M + kBM - 1) / kBM;
  const int tiles = NT * MT;

  if (warp == 0) tmem_alloc(tmem_slot, 2 * BN);
  if (warp == 1 && lane == 0) {
    for (int s = 0; s < NST; ++s) {
      mbar_init(&full[s], 1 + kProducers);  // the TMA thread + every producer thread
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    mbar_init(w2full, 1);
    mbar_init(a2full, 20 * 32);  // every epilogue and producer thread, once per round
    mbar_init(l2done, 1);
    fence_mbar_init();
  }
  if (warp == 2 && lane == 0) {
    tma_prefetch_desc(&tmBh);
    tma_prefetch_desc(&tmBl);
    tma_prefetch_desc(&tmYh);
    tma_prefetch_desc(&tmYl);
    if (L2) {
      tma_prefetch_desc(&l2.wh);
      tma_prefetch_desc(&l2.wl);
    }
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      uint32_t g = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
        const int n0 = (t % NT) * BN;
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % NST;
          const uint32_t ph = (g / NST) & 1;
          if (!mbar_wait(&empty[s], ph ^ 1, err)) {
            ok = false;
            break;
          }
          mbar_arrive_expect_tx(&full[s], 2 * C::B_BYTES);
          tma_load_2d(b_hi(s), &tmBh, kb * kBK, n0, &full[s]);
          tma_load_2d(b_lo(s), &tmBl, kb * kBK, n0, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_tf32_f32(kBM, BN);
      uint32_t g = 0;
      int i = 0;
      bool ok = true;
      for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x, ++i) {
        const int buf = i & 1;
        const uint32_t acc = tmem + static_cast<uint32_t>(buf * BN);
        if (!mbar_wait(&acc_empty[buf], ((i >> 1) & 1) ^ 1, err)) break;
        tc_fence_after();
        for (int kb = 0; kb < KB; ++kb, ++g) {
          const int s = g % NST;
          const uint32_t ph = (g / NST) & 1;
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
  } else if (warp < 6) {
    // ---- epilogue warps: layer 1's bias, ReLU, hi/lo planes (with L2, the layer-2
    // phase below consumes the accumulator instead)
    const int q = warp & 3;
    int i = 0;
    for (int t = blockIdx.x; t < (L2 ? 0 : tiles); t += gridDim.x, ++i) {
      const int buf = i & 1;
      const int m0 = (t / NT) * kBM, n0 = (t % NT) * BN;
      if (!mbar_wait(&acc_full[buf], (i >> 1) & 1, err)) break;
      tc_fence_after();
      const int row = m0 + q * 32 + lane;
      const uint32_t tm = tmem + static_cast<uint32_t>(buf * BN) + (static_cast<uint32_t>(q * 32) << 16);
      if (t + static_cast<int>(gridDim.x) >= tiles) {
        // the CTA's last tile: out through the idle stage ring and TMA stores, the
        // quarter's column blocks shared with its four producer warps (worker 0 of 5)
        tail_store_f32_planes<BN, 1>(tm, smem + (q * 5) * 8192, lane, b1, true, &tmYh, &tmYl, n0, m0 + q * 32,
                                     m0 + q * 32 < M, 0, 5);
        tc_fence_before();
        mbar_arrive(&acc_empty[buf]);
        continue;
      }
      const size_t ro = static_cast<size_t>(row < M ? row : 0) * ldy + n0;
#pragma unroll 1
      for (int c0 = 0; c0 < BN; c0 += 32) {
        uint32_t v[32];
        tmem_ld_32cols(tm + c0, v);
        tmem_ld_wait();
        if (row < M) {
          float4* dh = reinterpret_cast<float4*>(Yh + ro + c0);
          float4* dl = reinterpret_cast<float4*>(Yl + ro + c0);
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            float o[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) o[u] = fmaxf(__uint_as_float(v[4 * j + u]) + __ldg(b1 + n0 + c0 + 4 * j + u), 0.f);
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
      mbar_arrive(&acc_empty[buf]);
    }
  } else {
    // ---- producers: layer 0 for row pr of the tile, 32 columns per k-block, written
    // as the A tiles' hi/lo planes (row pr: 8 chunks of 16 B, chunk c at slot c ^ (pr % 8))
    const int pr = ((warp - 6) & 3) * 32 + lane;
    const int c0 = ((warp - 6) >> 2) * (8 / kGroups);
    // the row's dense features, padded: x[K0] = 1 multiplies the bias, the rest 0
    float x[kKM];
    auto load_x = [&](int t) {
      const int row = (t / NT) * kBM + pr;
#pragma unroll
      for (int k = 0; k < kKM; ++k) x[k] = k == K0 ? 1.f : 0.f;
      if (row < M) {
        const int inv = tab.n == 1 ? 0 : find_inv(tab, row);
        const float* dense = tab.d[inv].dense + static_cast<size_t>(row - tab.d[inv].row_base) * K0;
#pragma unroll
        for (int k = 0; k < kKM; ++k)
          if (k < K0) x[k] = __ldg(dense + k);
      }
    };
    if (static_cast<int>(blockIdx.x) < tiles) load_x(blockIdx.x);  // in flight during the staging
    {
      // layer 0's weights into rows of 16 -- weights, the bias (slot K0), zeros -- with
      // every load in flight before the first store; then wait for the producers only
      const int pt = threadIdx.x - 192;
      // W0 is [N0, K0] contiguous and 16-byte aligned: kV float4 per thread cover it,
      // then the biases (N0 / 4 float4) and the zero padding
      constexpr int kV = (kW0Max * (kKM - 1) / 4 + kProducers - 1) / kProducers;
      const int nv = N0 * K0 / 4;  // N0 is a multiple of 32, so N0 * K0 is a multiple of 4
      float4 wv[kV];
#pragma unroll
      for (int i = 0; i < kV; ++i)
        wv[i] = pt + i * kProducers < nv ? __ldg(reinterpret_cast<const float4*>(W0) + pt + i * kProducers)
                                         : make_float4(0.f, 0.f, 0.f, 0.f);
      const float4 bv = pt < N0 / 4 ? __ldg(reinterpret_cast<const float4*>(b0) + pt) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int i = 0; i < kV; ++i) {
        const int e4 = pt + i * kProducers;
        if (e4 < nv) {
          const float f[4] = {wv[i].x, wv[i].y, wv[i].z, wv[i].w};
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = 4 * e4 + u;
            sW0[(e / K0) * kKM + e % K0] = f[u];
          }
        }
      }
      if (pt < N0 / 4) {
        const float f[4] = {bv.x, bv.y, bv.z, bv.w};
#pragma unroll
        for (int u = 0; u < 4; ++u) sW0[(4 * pt + u) * kKM + K0] = f[u];
      }
      for (int e = pt; e < N0 * (kKM - 1 - K0); e += kProducers)
        sW0[(e / (kKM - 1 - K0)) * kKM + K0 + 1 + e % (kKM - 1 - K0)] = 0.f;
      named_barrier_sync(1, kProducers);
    }
    const uint32_t rbase = static_cast<uint32_t>((pr >> 3) * 1024 + (pr & 7) * 128);
    uint32_t g = 0;
    bool ok = true;
    for (int t = blockIdx.x; t < tiles && ok; t += gridDim.x) {
      if (t != static_cast<int>(blockIdx.x)) load_x(t);
      for (int kb = 0; kb < KB; ++kb, ++g) {
        const int s = g % NST;
        const uint32_t ph = (g / NST) & 1;
        if (!mbar_wait(&empty[s], ph ^ 1, err)) {
          ok = false;
          break;
        }
        uint8_t* ah = a_hi(s);
        uint8_t* al = a_lo(s);
#pragma unroll 2
        for (int c = c0; c < c0 + 8 / kGroups; ++c) {
          float h[4], l[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j = kb * kBK + c * 4 + u;
            const float4* wv = reinterpret_cast<const float4*>(sW0 + j * kKM);
            float acc = 0.f;
#pragma unroll
            for (int q = 0; q < kKM / 4; ++q) {
              const float4 w = wv[q];  // broadcast: every producer thread reads the same column
              acc = fmaf(x[4 * q], w.x, acc);
              acc = fmaf(x[4 * q + 1], w.y, acc);
              acc = fmaf(x[4 * q + 2], w.z, acc);
              acc = fmaf(x[4 * q + 3], w.w, acc);
            }
            const float y0 = fmaxf(acc, 0.f);
            h[u] = to_tf32_rna(y0);
            l[u] = y0 - h[u];
          }
          const uint32_t off = rbase + ((static_cast<uint32_t>(c) ^ static_cast<uint32_t>(pr & 7)) << 4);
          *reinterpret_cast<float4*>(ah + off) = make_float4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<float4*>(al + off) = make_float4(l[0], l[1], l[2], l[3]);
        }
        fence_proxy_async_smem();  // generic-proxy writes -> the tensor cores' reads
        mbar_arrive(&full[s]);
      }
      if (!L2 && ok && t + static_cast<int>(gridDim.x) >= tiles) {
        // the CTA's last tile: help the epilogue warp of this row quarter write it
        // (worker 1 + set of 5), once its MMAs have completed
        const int q = warp & 3, wk = 1 + ((warp - 6) >> 2);
        const int i = (t - static_cast<int>(blockIdx.x)) / static_cast<int>(gridDim.x);
        const int buf = i & 1;
        const int m0 = (t / NT) * kBM, n0 = (t % NT) * BN;
        if (!mbar_wait(&acc_full[buf], (i >> 1) & 1, err)) break;
        tc_fence_after();
        const uint32_t tm = tmem + static_cast<uint32_t>(buf * BN) + (static_cast<uint32_t>(q * 32) << 16);
        tail_store_f32_planes<BN, 1>(tm, smem + (q * 5 + wk) * 8192, lane, b1, true, &tmYh, &tmYl, n0,
                                     m0 + q * 32, m0 + q * 32 < M, wk, 5);
      }
    }
  }
  if constexpr (L2) {
    if (static_cast<int>(blockIdx.x) < tiles) {
      const int N2 = l2.n;
      constexpr int KB2 = BN / kBK;  // layer 2 reduces over layer 1's BN = N1 outputs
      const int w2kb = N2 * kBK * 4;  // one plane of a W2 k-block
      const int h = min(KB2, (NST * C::STAGE) / (2 * C::A_BYTES + 2 * w2kb));
      const int R = (KB2 + h - 1) / h;
      uint8_t* a2 = smem;                         // h slots: A hi, A lo (16 KB each)
      uint8_t* w2 = smem + h * 2 * C::A_BYTES;  // h slots: W2 hi, W2 lo
      const int m0 = blockIdx.x * kBM;
      bool ok = true;
      if (warp == 0) {
        if (lane == 0) {
          // the W2 slots overlap the stage ring: wait until layer 1's MMAs have read it
          ok = mbar_wait(&acc_full[0], 0, err);
          for (int r = 0; r < R && ok; ++r) {
            if (r > 0 && !mbar_wait(l2done, (r - 1) & 1, err)) break;  // the previous round's reads
            const int k0 = r * h, k1 = min(KB2, k0 + h);
            mbar_arrive_expect_tx(w2full, static_cast<uint32_t>((k1 - k0) * 2 * w2kb));
            for (int kb = k0; kb < k1; ++kb) {
              uint8_t* dst = w2 + (kb - k0) * 2 * w2kb;
              tma_load_2d(dst, &l2.wh, kb * kBK, 0, w2full);
              tma_load_2d(dst + w2kb, &l2.wl, kb * kBK, 0, w2full);
            }
          }
        }
      } else if (warp == 1) {
        if (lane == 0) {
          const uint32_t idesc2 = idesc_tf32_f32(kBM, N2);
          const uint32_t acc2 = tmem + BN;
          for (int r = 0; r < R && ok; ++r) {
            if (!mbar_wait(w2full, r & 1, err) || !mbar_wait(a2full, r & 1, err)) break;
            tc_fence_after();
            const int k0 = r * h, k1 = min(KB2, k0 + h);
            for (int kb = k0; kb < k1; ++kb) {
              const uint32_t ah = smem_u32(a2 + (kb - k0) * 2 * C::A_BYTES), al = ah + C::A_BYTES;
              const uint32_t bh = smem_u32(w2 + (kb - k0) * 2 * w2kb), bl = bh + w2kb;
#pragma unroll
              for (int k = 0; k < kBK / 8; ++k) {
                const uint32_t o = k * 32;
                tc_mma_tf32_fill_a(acc2, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bh + o), idesc2,
                                   (kb | k) != 0 ? 1u : 0u);
                tc_mma_tf32_lastuse_a(acc2, sw128_kmajor_desc(ah + o), sw128_kmajor_desc(bl + o), idesc2, 1u);
                tc_mma_tf32(acc2, sw128_kmajor_desc(al + o), sw128_kmajor_desc(bh + o), idesc2, 1u);
              }
            }
            tc_commit(l2done);
          }
        }
      } else {
        // workers: per row quarter q the epilogue warp (wk 0) and four producer warps
        // (wk 1..4) share the 32-column blocks, as in the last-tile output above
        const int q = warp & 3, wk = warp < 6 ? 0 : 1 + ((warp - 6) >> 2);
        const uint32_t lanes = static_cast<uint32_t>(q * 32) << 16;
        const int ar = q * 32 + lane;  // this thread's row of the A tiles
        ok = mbar_wait(&acc_full[0], 0, err);
        tc_fence_after();
        for (int r = 0; r < R && ok; ++r) {
          if (r > 0 && !mbar_wait(l2done, (r - 1) & 1, err)) {
            ok = false;
            break;
          }
          const int k0 = r * h, k1 = min(KB2, k0 + h);
          for (int kb = k0 + wk; kb < k1; kb += 5) {
            uint32_t v[32];
            tmem_ld_32cols(tmem + lanes + kb * kBK, v);
            tmem_ld_wait();
            uint8_t* ah = a2 + (kb - k0) * 2 * C::A_BYTES;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              float o[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) o[u] = fmaxf(__uint_as_float(v[4 * j + u]) + __ldg(b1 + kb * kBK + 4 * j + u), 0.f);
              float4 hv, lv;
              hv.x = to_tf32_rna(o[0]);
              hv.y = to_tf32_rna(o[1]);
              hv.z = to_tf32_rna(o[2]);
              hv.w = to_tf32_rna(o[3]);
              lv.x = o[0] - hv.x;
              lv.y = o[1] - hv.y;
              lv.z = o[2] - hv.z;
              lv.w = o[3] - hv.w;
              const uint32_t off = static_cast<uint32_t>(ar * 128 + ((j ^ (ar & 7)) << 4));
              *reinterpret_cast<float4*>(ah + off) = hv;
              *reinterpret_cast<float4*>(ah + C::A_BYTES + off) = lv;
            }
          }
          fence_proxy_async_smem();
          mbar_arrive(a2full);
        }
        // layer 2's output (bias, ReLU, hi/lo planes) once the last round's MMAs completed
        if (ok && mbar_wait(l2done, (R - 1) & 1, err)) {
          tc_fence_after();
          tail_store_f32_planes<256, 1>(tmem + BN + lanes, smem + (q * 5 + wk) * 8192, lane, l2.b, true, &tmYh,
                                        &tmYl, 0, m0 + q * 32, m0 + q * 32 < M, wk, 5, N2);
        }
      }
    }
  }
  __syncwarp();
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * BN);
}

// yh / yl / ldy: layer 1's output, or layer 2's when `w2h` is given (N2 outputs).
template <int BN, int NST, bool L2>
cudaError_t launch_b01(const InvTable& tab, int K0, int N0, const float* W0, const float* b0, int N1,
                       const float* w1h, const float* w1l, const float* b1, float* yh, float* yl, int ldy, int* err,
                       cudaStream_t s, const float* w2h, const float* w2l, const float* b2, int N2) {
  static DeviceOnce once;
  if (cudaError_t e = device_once(once, [](int) {
        return cudaFuncSetAttribute(bottom01_kernel<BN, NST, L2>,
                                    cudaFuncAttributeMaxDynamicSharedMemorySize, B01Cfg<BN, NST>::SMEM);
      });
      e != cudaSuccess)
    return e;
  const int nout = L2 ? N2 : N1;
  CUtensorMap tbh, tbl, tyh, tyl;
  Layer2 l2{};
  if (!make_tmap_2d(&tbh, 0, w1h, N1, N0, N0, kBK, BN) || !make_tmap_2d(&tbl, 0, w1l, N1, N0, N0, kBK, BN) ||
      !make_tmap_2d(&tyh, 0, yh, tab.M, nout, ldy, 32, 32) || !make_tmap_2d(&tyl, 0, yl, tab.M, nout, ldy, 32, 32))
    return cudaErrorInvalidValue;
  const int tiles = (N1 / BN) * ((tab.M + kBM - 1) / kBM);
  if (L2) {
    if (BN != N1 || tiles > device_sms()) return cudaErrorInvalidValue;  // one whole-row tile per CTA
    if (!make_tmap_2d(&l2.wh, 0, w2h, N2, N1, N1, kBK, N2) || !make_tmap_2d(&l2.wl, 0, w2l, N2, N1, N1, kBK, N2))
      return cudaErrorInvalidValue;
    l2.b = b2;
    l2.n = N2;
  }
  const int sms_n = device_sms();
  const int grid = tiles < sms_n ? tiles : sms_n;
  bottom01_kernel<BN, NST, L2><<<grid, kThreads, B01Cfg<BN, NST>::SMEM, s>>>(
      tbh, tbl, tyh, tyl, tab, K0, N0, W0, b0, N1, b1, yh, yl, ldy, err, l2);
  count_launch();
  return cudaGetLastError();
}

}  // namespace

bool bottom01_fusable(int K0, int N0, int N1) {
  return K0 >= 1 && K0 < kKM && N0 >= kBK && N0 <= kW0Max && N0 % kBK == 0 && N1 % 64 == 0;
}

// Tile configurations: (BN, stages + 100), all persistent; BN = N1 computes layer 0
// once per row, narrower tiles recompute it for each of the N1 / BN column tiles.
// (256, 202): the same tile, and layer 2 computed in the kernel too.
const GemmCfg kB01Cfgs[] = {{256, 102}, {128, 103}, {64, 104}, {256, 202}};

int bottom01_candidates(GemmCfg* out, int max) {
  int n = 0;
  for (const GemmCfg& c : kB01Cfgs)
    if (n < max) out[n++] = c;
  if (n < max) out[n++] = GemmCfg{1, 1};  // separate kernels
  return n;
}

bool bottom012_fusable(int N1, int N2, int M) {
  return N1 == 256 && N2 >= 32 && N2 <= 256 && N2 % 32 == 0 && (M + kBM - 1) / kBM <= device_sms();
}

GemmCfg bottom01_default(int N1) {
  if (N1 % 256 == 0 && N1 <= 256) return GemmCfg{256, 102};
  if (N1 % 128 == 0) return GemmCfg{128, 103};
  return GemmCfg{64, 104};
}

cudaError_t launch_bottom01_f32(const InvTable& tab, int K0, int N0, const float* W0, const float* b0, int N1,
                                const float* w1h, const float* w1l, const float* b1, float* yh, float* yl, int ldy,
                                int* err, cudaStream_t s, GemmCfg cfg, const float* w2h, const float* w2l,
                                const float* b2, int N2, int* layers) {
  const bool three = w2h && w2l && b2 && bottom012_fusable(N1, N2, tab.M);
  if (cfg.bn == 0) cfg = three ? GemmCfg{256, 202} : bottom01_default(N1);
  if (cfg.stages == 202 && !three) cfg = GemmCfg{256, 102};  // layer 2 then runs separately
  if (layers) *layers = cfg.stages == 202 ? 3 : 2;
  if (tab.M <= 0) return cudaSuccess;
  if (!bottom01_fusable(K0, N0, N1) || (ldy % 4)) return cudaErrorInvalidValue;
  for (const void* p : {static_cast<const void*>(w1h), static_cast<const void*>(w1l), static_cast<const void*>(yh),
                        static_cast<const void*>(yl), static_cast<const void*>(W0), static_cast<const void*>(b0),
                        static_cast<const void*>(w2h), static_cast<const void*>(w2l)})
    if (reinterpret_cast<uintptr_t>(p) & 15) return cudaErrorInvalidValue;
  if (N1 % cfg.bn) return cudaErrorInvalidValue;
  if (cfg.bn == 256 && cfg.stages == 202) {
    return launch_b01<256, 2, true>(tab, K0, N0, W0, b0, N1, w1h, w1l, b1, yh, yl, ldy, err, s, w2h, w2l, b2, N2);
  }
  if (cfg.bn == 256 && cfg.stages == 102)
    return launch_b01<256, 2, false>(tab, K0, N0, W0, b0, N1, w1h, w1l, b1, yh, yl, ldy, err, s, nullptr, nullptr,
                                     nullptr, 0);
  if (cfg.bn == 128 && cfg.stages == 103)
    return launch_b01<128, 3, false>(tab, K0, N0, W0, b0, N1, w1h, w1l, b1, yh, yl, ldy, err, s, nullptr, nullptr,
                                     nullptr, 0);
  if (cfg.bn == 64 && cfg.stages == 104)
    return launch_b01<64, 4, false>(tab, K0, N0, W0, b0, N1, w1h, w1l, b1, yh, yl, ldy, err, s, nullptr, nullptr,
                                    nullptr, 0);
  return cudaErrorInvalidValue;
}

void preload_bottom01_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, bottom01_kernel<256, 2, false>);
  cudaFuncGetAttributes(&fa, bottom01_kernel<256, 2, true>);
  cudaFuncGetAttributes(&fa, bottom01_kernel<128, 3, false>);
  cudaFuncGetAttributes(&fa, bottom01_kernel<64, 4, false>);
}

}  // namespace sage
