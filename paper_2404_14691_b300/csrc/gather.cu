// Embedding-bag gather-sum over a fused batch of invocations (HBM-bound).
//
// Each warp owns one bag at a time (the T*M bags of the batch in table-major order,
// so that neighbouring warps read the same table; a warp's bags are a fixed
// grid-stride share, or -- with GatherArgs::work -- claimed from a counter as it
// goes, which balances bags of uneven length and lets blocks that start early take
// more).  A row of the
// table is LPR lanes x 16 bytes; a warp therefore reads RPW = 32/LPR rows per
// load instruction and keeps U such instructions in flight.  Row indices are
// fetched 32 at a time with one coalesced load and broadcast with shuffles.
// Sub-group s of the warp sums the bag positions p with p % RPW == s in position
// order; the RPW partial sums are then combined by a fixed xor tree.  The order
// of every sum therefore depends only on the bag itself, never on the batch it
// runs in, which makes fused and isolated invocations bitwise identical.
#include <algorithm>
#include <type_traits>

#include "kernels.h"

namespace sage {
namespace {

template <int N>
struct Acc {
  float v[N];
};

__device__ __forceinline__ uint4 ldg_nc_v4(const uint4* p) { return __ldg(p); }

// The warp's next unit of work from the launch's `next` counter (called by all lanes).
__device__ __forceinline__ uint32_t claim(unsigned* work) {
  uint32_t q = 0;
  if ((threadIdx.x & 31) == 0) q = atomicAdd(work, 1u);
  return __shfl_sync(0xffffffffu, q, 0);
}

// End of a block that claimed work: the grid's last block to get here -- every other
// block has made its final claim by then -- resets both counters for the next launch.
__device__ __forceinline__ void block_done(unsigned* work) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(work + 1, 1u) == gridDim.x - 1) {
      atomicExch(work, 0u);
      atomicExch(work + 1, 0u);
    }
  }
}

// acc + the bf16 in the low / high half of w, one fp32 rounding: the mixed-precision
// add converts the bf16 exactly and adds it to the fp32 accumulator, as unpacking it
// to fp32 and adding would, without the unpacking instruction.
__device__ __forceinline__ float add_bf16_lo(uint32_t w, float acc) {
  float r;
  asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tadd.rn.f32.bf16 %0, l, %2;\n\t}" : "=f"(r) : "r"(w), "f"(acc));
  return r;
}
__device__ __forceinline__ float add_bf16_hi(uint32_t w, float acc) {
  float r;
  asm("{\n\t.reg .b16 l, h;\n\tmov.b32 {l, h}, %1;\n\tadd.rn.f32.bf16 %0, h, %2;\n\t}" : "=f"(r) : "r"(w), "f"(acc));
  return r;
}


// acc += one 16-byte vector of a row (bf16: 8 elements, element 2e the low half of
// word e; fp32: 4 elements), one round-to-nearest fp32 addition per element.
template <bool BF16>
__device__ __forceinline__ void accumulate(float* acc, const uint4& v) {
  if (BF16) {
    const uint32_t wd[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      acc[2 * e] = add_bf16_lo(wd[e], acc[2 * e]);
      acc[2 * e + 1] = add_bf16_hi(wd[e], acc[2 * e + 1]);
    }
  } else {
    // two independent round-to-nearest adds per instruction, as four scalar adds would
    asm("{\n\t.reg .b64 a, b;\n\tmov.b64 a, {%0, %1};\n\tmov.b64 b, {%4, %5};\n\t"
        "add.rn.f32x2 a, a, b;\n\tmov.b64 {%0, %1}, a;\n\t"
        "mov.b64 a, {%2, %3};\n\tmov.b64 b, {%6, %7};\n\tadd.rn.f32x2 a, a, b;\n\tmov.b64 {%2, %3}, a;\n\t}"
        : "+f"(acc[0]), "+f"(acc[1]), "+f"(acc[2]), "+f"(acc[3])
        : "f"(__uint_as_float(v.x)), "f"(__uint_as_float(v.y)), "f"(__uint_as_float(v.z)), "f"(__uint_as_float(v.w)));
  }
}

// Combine the 32 / LPR sub-group partial sums of a bag (fixed xor tree; a + b == b + a
// exactly) and write the pooled row (bf16, fp32, or fp32 as tf32 hi / residual lo).
template <bool BF16, int LPR, int VPL>
__device__ __forceinline__ void finish_bag(float (&acc)[VPL][BF16 ? 8 : 4], const GatherArgs& a, int t, int r,
                                           int sub, int col) {
  constexpr int EPV = BF16 ? 8 : 4;
#pragma unroll
  for (int o = LPR; o < 32; o <<= 1)
#pragma unroll
    for (int w = 0; w < VPL; ++w)
#pragma unroll
      for (int e = 0; e < EPV; ++e) acc[w][e] += __shfl_xor_sync(0xffffffffu, acc[w][e], o);
  if (sub != 0) return;
  char* orow = static_cast<char*>(a.out) +
               (static_cast<size_t>(r) * a.ldo + static_cast<size_t>(t) * a.dim) * (BF16 ? 2 : 4);
#pragma unroll
  for (int w = 0; w < VPL; ++w) {
    uint4 o;
    if (BF16) {
      o.x = pack_bf16x2(acc[w][0], acc[w][1]);
      o.y = pack_bf16x2(acc[w][2], acc[w][3]);
      o.z = pack_bf16x2(acc[w][4], acc[w][5]);
      o.w = pack_bf16x2(acc[w][6], acc[w][7]);
    } else if (a.out_lo) {
      // hi/lo planes for the fp32 tensor-core layers: hi = tf32(sum), lo = sum - hi
      float h[4], l[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        h[e] = to_tf32_rna(acc[w][e]);
        l[e] = acc[w][e] - h[e];
      }
      o = make_uint4(__float_as_uint(h[0]), __float_as_uint(h[1]), __float_as_uint(h[2]), __float_as_uint(h[3]));
      float* lrow = a.out_lo + static_cast<size_t>(r) * a.ldo + static_cast<size_t>(t) * a.dim;
      reinterpret_cast<float4*>(lrow)[col + w * LPR] = make_float4(l[0], l[1], l[2], l[3]);
    } else {
      o = make_uint4(__float_as_uint(acc[w][0]), __float_as_uint(acc[w][1]), __float_as_uint(acc[w][2]),
                     __float_as_uint(acc[w][3]));
    }
    reinterpret_cast<uint4*>(orow)[col + w * LPR] = o;
  }
}

// Walk runs of `run` (<= RUN) consecutive bags (table-major: consecutive rows of one
// table, moving to the next table after row M - 1), claimed one run at a time from
// `work` or, without it (or beyond 32-bit bag arithmetic), as a fixed grid-stride
// share, calling bag_sum(t, r, i) for table t, batch row r of invocation i.  Inside a run the table,
// the row and its invocation advance incrementally, so the division and the
// invocation search happen once per run; 32-bit index arithmetic whenever the bag
// count allows it (a 64-bit division is a long instruction sequence).  RUN = 1
// compiles to one bag per step, without the run's extra live registers.
template <int RUN, class F>
__device__ __forceinline__ void walk_bags(const InvTable& tab, int T, int run, unsigned* work, F&& bag_sum) {
  const int64_t G = static_cast<int64_t>(T) * tab.M;
  const int64_t nwarps = (static_cast<int64_t>(gridDim.x) * blockDim.x) >> 5;
  auto walk = [&](int t, int r, int cnt) {
    int i = tab.n == 1 ? 0 : find_inv(tab, r);
    if constexpr (RUN == 1) {
      bag_sum(t, r, i);
    } else {
      for (int k = 0;;) {
        bag_sum(t, r, i);
        if (++k == cnt) break;
        if (++r == tab.M) {
          r = 0;
          ++t;
          i = 0;
        }
        while (i + 1 < tab.n && tab.d[i + 1].row_base <= r) ++i;
      }
    }
  };
  const int64_t first = (static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const int64_t runs = (G + run - 1) / run;
  if (G + nwarps * run < (int64_t(1) << 32)) {
    const uint32_t M = static_cast<uint32_t>(tab.M), G32 = static_cast<uint32_t>(G);
    const uint32_t step = static_cast<uint32_t>(nwarps), R32 = static_cast<uint32_t>(runs);
    if (work) {
      // claimed runs (one bag each for RUN = 1)
      for (;;) {
        const uint32_t q = claim(work);
        if (q >= R32) break;
        const uint32_t g0 = q * static_cast<uint32_t>(run);
        const uint32_t t = g0 / M;
        walk(static_cast<int>(t), static_cast<int>(g0 - t * M),
             static_cast<int>(min(static_cast<uint32_t>(run), G32 - g0)));
      }
    } else if constexpr (RUN == 1) {
      // one bag per step: the table and row advance by the grid's warp count without a division
      uint32_t g = static_cast<uint32_t>(first);
      uint32_t t = g / M, r = g - t * M;
      const uint32_t dt = step / M, dr = step - dt * M;
      for (; g < G32; g += step) {
        walk(static_cast<int>(t), static_cast<int>(r), 1);
        t += dt;
        r += dr;
        if (r >= M) {
          r -= M;
          ++t;
        }
      }
    } else {
      for (uint32_t q = static_cast<uint32_t>(first); q < R32; q += step) {
        const uint32_t g0 = q * static_cast<uint32_t>(run);
        const uint32_t t = g0 / M;
        walk(static_cast<int>(t), static_cast<int>(g0 - t * M),
             static_cast<int>(min(static_cast<uint32_t>(run), G32 - g0)));
      }
    }
  } else {
    for (int64_t q = first; q < runs; q += nwarps) {
      const int64_t g0 = q * run;
      const int t = static_cast<int>(g0 / tab.M);
      walk(t, static_cast<int>(g0 - static_cast<int64_t>(t) * tab.M), static_cast<int>(G - g0 < run ? G - g0 : run));
    }
  }
}

// One step of a bag: UU row loads in flight per lane, bag positions q + u*RPW + sub of
// the current 32-index chunk (row indices in lane p of `my`); the position check is
// needed only in a bag's last, partial steps.  Rows out of the table's range set the
// bounds error bit and are skipped.
template <bool BF16, int LPR, int VPL, int UU, bool CHECKED>
__device__ __forceinline__ void bag_step(float (&acc)[VPL][BF16 ? 8 : 4], const GatherArgs& a, const char* base,
                                         unsigned rows, int sub, int col, int q, int cnt, int my) {
  constexpr int RPW = 32 / LPR;
  constexpr unsigned kRowBytes = LPR * VPL * 16;  // a row is LPR lanes x VPL x 16 bytes
  const char* lane_base = base + col * 16;
  uint4 v[UU][VPL];
  unsigned row[UU];
#pragma unroll
  for (int u = 0; u < UU; ++u) row[u] = static_cast<unsigned>(__shfl_sync(0xffffffffu, my, (q + u * RPW + sub) & 31));
  if constexpr (!CHECKED) {
    // all UU positions lie in the bag: one range check for the step, the rare
    // out-of-range step takes the checked path below
    unsigned hi = row[0];
#pragma unroll
    for (int u = 1; u < UU; ++u) hi = max(hi, row[u]);
    if (hi < rows) {
#pragma unroll
      for (int u = 0; u < UU; ++u) {
        const uint4* src = reinterpret_cast<const uint4*>(lane_base + static_cast<uint64_t>(row[u]) * kRowBytes);
#pragma unroll
        for (int w = 0; w < VPL; ++w) v[u][w] = ldg_nc_v4(src + w * LPR);
      }
#pragma unroll
      for (int u = 0; u < UU; ++u)
#pragma unroll
        for (int w = 0; w < VPL; ++w) accumulate<BF16>(acc[w], v[u][w]);
      return;
    }
  }
  bool ok[UU];
#pragma unroll
  for (int u = 0; u < UU; ++u) {
    ok[u] = CHECKED ? q + u * RPW + sub < cnt : true;
    if (ok[u] && row[u] >= rows) {
      ok[u] = false;
      if (a.err) atomicOr(a.err, kErrBounds);
    }
    const uint4* src = reinterpret_cast<const uint4*>(lane_base + static_cast<uint64_t>(ok[u] ? row[u] : 0u) * kRowBytes);
#pragma unroll
    for (int w = 0; w < VPL; ++w) v[u][w] = ok[u] ? ldg_nc_v4(src + w * LPR) : make_uint4(0, 0, 0, 0);
  }
#pragma unroll
  for (int u = 0; u < UU; ++u) {
    if (!ok[u]) continue;
#pragma unroll
    for (int w = 0; w < VPL; ++w) accumulate<BF16>(acc[w], v[u][w]);
  }
}

template <bool BF16, int LPR, int VPL, int U, int RUN>
__global__ void __launch_bounds__(256) gather_kernel(const __grid_constant__ GatherArgs a,
                                                     const __grid_constant__ InvTable tab, int run) {
  constexpr int RPW = 32 / LPR;
  constexpr int EPV = BF16 ? 8 : 4;  // elements per 16-byte vector
  const int lane = threadIdx.x & 31;
  const int sub = lane / LPR;
  const int col = lane % LPR;

  // bag (t, r): table t, batch row r of invocation i
  auto bag_sum = [&](int t, int r, int i) {
    const InvDesc& d = tab.d[i];
    const int64_t bag = static_cast<int64_t>(t) * d.batch + (r - d.row_base);
    const int64_t beg = d.offsets[bag];
    const int64_t end = d.offsets[bag + 1];
    const char* base = a.tables + a.table_off[t];
    const unsigned rows = static_cast<unsigned>(a.table_rows[t]);

    // running fp32 sums, one per element: bf16 elements added by mixed-precision adds
    // (element 2e is the low half of word e), fp32 elements by plain adds; either way
    // each element gets the same sequence of round-to-nearest fp32 additions.
    float acc[VPL][EPV];
#pragma unroll
    for (int w = 0; w < VPL; ++w) {
#pragma unroll
      for (int e = 0; e < EPV; ++e) acc[w][e] = 0.f;
    }

    // tail steps: fewer loads per step, fewer idle slots; 4 for bf16 256-byte rows (2 or 8
    // were slower there), 2 elsewhere
    constexpr int UT = BF16 && LPR == 16 ? 4 : (U < 2 ? U : 2);
    for (int64_t j0 = beg; j0 < end; j0 += 32) {
      const int cnt = static_cast<int>(min(static_cast<int64_t>(32), end - j0));
      const int my = lane < cnt ? __ldg(d.indices + j0 + lane) : 0;
      int q = 0;
      // each lane still adds its positions in increasing order: same sums as one loop
      for (; q + RPW * U <= cnt; q += RPW * U)
        bag_step<BF16, LPR, VPL, U, false>(acc, a, base, rows, sub, col, q, cnt, my);
      for (; q < cnt; q += RPW * UT) bag_step<BF16, LPR, VPL, UT, true>(acc, a, base, rows, sub, col, q, cnt, my);
    }
    finish_bag<BF16, LPR, VPL>(acc, a, t, r, sub, col);
  };
  walk_bags<RUN>(tab, a.T, run, a.work, bag_sum);
  if (a.work) block_done(a.work);
}

template <bool BF16, int LPR, int VPL, int U, int RUN>
cudaError_t launch_one(const GatherArgs& a, const InvTable& tab, cudaStream_t s) {
  // per device: the largest L1 carve-out (no shared memory is used) and the occupancy
  static DeviceOnce once;
  static int bps[kMaxDevices];
  int dev = 0;
  if (cudaError_t e = device_once(
          once,
          [](int d) {
            cudaFuncSetAttribute(gather_kernel<BF16, LPR, VPL, U, RUN>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxL1);
            int b = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gather_kernel<BF16, LPR, VPL, U, RUN>, 256, 0);
            bps[d] = b < 1 ? 1 : b;
            return cudaSuccess;
          },
          &dev);
      e != cudaSuccess)
    return e;
  const int blocks_per_sm = bps[dev], sms = device_sms();
  const int64_t bags = static_cast<int64_t>(a.T) * tab.M;
  if (bags == 0) return cudaSuccess;
  // runs of up to RUN bags per warp once there are several bags per resident warp;
  // small batches keep one bag per warp, for parallelism
  const int64_t resident = static_cast<int64_t>(sms) * blocks_per_sm * 8;
  const int run = static_cast<int>(std::max<int64_t>(1, std::min<int64_t>(RUN, bags / (4 * resident))));
  int64_t need = ((bags + run - 1) / run + 7) / 8;
  int64_t grid = static_cast<int64_t>(sms) * blocks_per_sm;
  if (need < grid) grid = need;
  gather_kernel<BF16, LPR, VPL, U, RUN><<<static_cast<unsigned>(grid), 256, 0, s>>>(a, tab, run);
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------- bag per lane group
//
// For short bags the per-bag work (invocation, offsets, table base, the sub-group
// combine, the output) outweighs the row loads.  Here a warp's 32 / LPR lane groups
// each own a bag: the per-bag work runs once for all of them, in the same
// instructions, and no combine is needed.  A group reads its bag's rows one at a
// time (LPR lanes x VPL x 16 bytes = one row), U rows in flight, and each lane adds
// its pieces in bag order: one fixed order per bag, whatever the batch.  The warp
// loops to the longest of its bags; the other groups' lanes idle meanwhile.
template <bool BF16, int LPR, int VPL, int U>
__global__ void __launch_bounds__(256) gather_group_kernel(const __grid_constant__ GatherArgs a,
                                                           const __grid_constant__ InvTable tab) {
  constexpr int NG = 32 / LPR;
  constexpr int EPV = BF16 ? 8 : 4;
  const int lane = threadIdx.x & 31;
  const int grp = lane / LPR;
  const int gl = lane % LPR;
  const uint32_t M = static_cast<uint32_t>(tab.M), T = static_cast<uint32_t>(a.T);
  const uint32_t slots = ((gridDim.x * blockDim.x) >> 5) * NG;  // bags per grid step
  const uint32_t first = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * NG + grp;
  const size_t row_bytes = static_cast<size_t>(a.dim) * (BF16 ? 2 : 4);
  // table and row of this group's bag: claimed NG bags at a time, or advanced by `slots`
  // bags per step without a division
  uint32_t t, r;
  if (a.work) {
    const uint32_t g = claim(a.work) * NG + grp;
    t = g / M;
    r = g - t * M;
  } else {
    t = first / M;
    r = first - t * M;
  }
  const uint32_t dt = slots / M, dr = slots - dt * M;
  while (__any_sync(0xffffffffu, t < T)) {
    int64_t beg = 0, end = 0;
    const char* base = a.tables;
    const int32_t* idx = nullptr;
    unsigned rows = 0;
    if (t < T) {
      const int i = tab.n == 1 ? 0 : find_inv(tab, static_cast<int>(r));
      const InvDesc& d = tab.d[i];
      const int64_t bag = static_cast<int64_t>(t) * d.batch + (static_cast<int>(r) - d.row_base);
      beg = d.offsets[bag];
      end = d.offsets[bag + 1];
      base = a.tables + a.table_off[t] + gl * (VPL * 16);
      rows = static_cast<unsigned>(a.table_rows[t]);
      idx = d.indices + beg;
    }
    const int len = static_cast<int>(end - beg);
    int maxlen = len;
#pragma unroll
    for (int o = LPR; o < 32; o <<= 1) maxlen = max(maxlen, __shfl_xor_sync(0xffffffffu, maxlen, o));
    float acc[VPL][EPV];
#pragma unroll
    for (int w = 0; w < VPL; ++w)
#pragma unroll
      for (int e = 0; e < EPV; ++e) acc[w][e] = 0.f;
    // the group's next CH * LPR indices, CH loads per lane issued together: index
    // position j0 + m * LPR + gl sits in lane gl's register m
    constexpr int CH = 32 / LPR;
    static_assert(U <= LPR && LPR % U == 0, "a step stays within one index register");
    for (int j0 = 0; j0 < maxlen; j0 += CH * LPR) {
      int my[CH];
#pragma unroll
      for (int m = 0; m < CH; ++m) my[m] = j0 + m * LPR + gl < len ? __ldg(idx + j0 + m * LPR + gl) : 0;
      const int cnt = min(CH * LPR, maxlen - j0);
      for (int p = 0; p < cnt; p += U) {
        uint4 v[U][VPL];
        bool ok[U];
        const int mp = p / LPR;  // the register holding positions p .. p + U - 1
        int src = my[0];
#pragma unroll
        for (int m = 1; m < CH; ++m) src = mp == m ? my[m] : src;
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int q = p + u;
          const int row = __shfl_sync(0xffffffffu, src, grp * LPR + (q & (LPR - 1)));
          ok[u] = q < cnt && j0 + q < len;
          if (ok[u] && static_cast<unsigned>(row) >= rows) {
            ok[u] = false;
            if (a.err) atomicOr(a.err, kErrBounds);
          }
          const uint4* src = reinterpret_cast<const uint4*>(base + static_cast<size_t>(ok[u] ? row : 0) * row_bytes);
#pragma unroll
          for (int w = 0; w < VPL; ++w) v[u][w] = ok[u] ? ldg_nc_v4(src + w) : make_uint4(0, 0, 0, 0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          if (!ok[u]) continue;
#pragma unroll
          for (int w = 0; w < VPL; ++w) accumulate<BF16>(acc[w], v[u][w]);
        }
      }
    }
    if (t < T) {
      // the group's pooled row: lane gl holds elements [gl * VPL * EPV, ...)
      const size_t o = static_cast<size_t>(r) * a.ldo + static_cast<size_t>(t) * a.dim;
#pragma unroll
      for (int w = 0; w < VPL; ++w) {
        uint4 ov;
        if (BF16) {
          ov.x = pack_bf16x2(acc[w][0], acc[w][1]);
          ov.y = pack_bf16x2(acc[w][2], acc[w][3]);
          ov.z = pack_bf16x2(acc[w][4], acc[w][5]);
          ov.w = pack_bf16x2(acc[w][6], acc[w][7]);
          reinterpret_cast<uint4*>(static_cast<__nv_bfloat16*>(a.out) + o)[gl * VPL + w] = ov;
        } else if (a.out_lo) {
          float h[4], l[4];
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            h[e] = to_tf32_rna(acc[w][e]);
            l[e] = acc[w][e] - h[e];
          }
          reinterpret_cast<float4*>(static_cast<float*>(a.out) + o)[gl * VPL + w] = make_float4(h[0], h[1], h[2], h[3]);
          reinterpret_cast<float4*>(a.out_lo + o)[gl * VPL + w] = make_float4(l[0], l[1], l[2], l[3]);
        } else {
          reinterpret_cast<float4*>(static_cast<float*>(a.out) + o)[gl * VPL + w] =
              make_float4(acc[w][0], acc[w][1], acc[w][2], acc[w][3]);
        }
      }
    }
    if (a.work) {
      const uint32_t g = claim(a.work) * NG + grp;
      t = g / M;
      r = g - t * M;
    } else {
      t += dt;
      r += dr;
      if (r >= M) {
        r -= M;
        ++t;
      }
    }
  }
  if (a.work) block_done(a.work);
}

template <bool BF16, int LPR, int VPL, int U>
cudaError_t launch_group(const GatherArgs& a, const InvTable& tab, cudaStream_t s) {
  // per device: the largest L1 carve-out (no shared memory is used) and the occupancy
  static DeviceOnce once;
  static int bps[kMaxDevices];
  int dev = 0;
  if (cudaError_t e = device_once(
          once,
          [](int d) {
            cudaFuncSetAttribute(gather_group_kernel<BF16, LPR, VPL, U>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxL1);
            int b = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, gather_group_kernel<BF16, LPR, VPL, U>, 256, 0);
            bps[d] = b < 1 ? 1 : b;
            return cudaSuccess;
          },
          &dev);
      e != cudaSuccess)
    return e;
  const int blocks_per_sm = bps[dev], sms = device_sms();
  constexpr int NG = 32 / LPR;
  const int64_t bags = static_cast<int64_t>(a.T) * tab.M;
  if (bags == 0) return cudaSuccess;
  int64_t need = (bags + 8 * NG - 1) / (8 * NG);
  int64_t grid = static_cast<int64_t>(sms) * blocks_per_sm;
  if (need < grid) grid = need;
  // 32-bit bag arithmetic: a warp's last claim (or grid-stride step) ends at most one
  // unit of NG bags beyond the grid's warps' share past the last bag
  if (bags + (grid * 8 + 1) * NG >= (int64_t(1) << 32)) return cudaErrorInvalidValue;
  gather_group_kernel<BF16, LPR, VPL, U><<<static_cast<unsigned>(grid), 256, 0, s>>>(a, tab);
  count_launch();
  return cudaGetLastError();
}

template <bool BF16>
cudaError_t dispatch(const GatherArgs& a, const InvTable& tab, cudaStream_t s) {
  const int rb = a.dim * (BF16 ? 2 : 4);
  switch (rb) {
    case 16: return launch_one<BF16, 1, 1, 1, 1>(a, tab, s);
    case 32: return launch_one<BF16, 2, 1, 1, 1>(a, tab, s);
    case 64: return launch_one<BF16, 4, 1, 2, 1>(a, tab, s);
    case 128: return launch_one<BF16, 8, 1, 4, BF16 ? 4 : 1>(a, tab, s);
    // 256-byte rows: fp32 as 8 lanes x 32 B per row, one bag per 8-lane group (short
    // bags: the per-bag work dominates; one bag per warp only for batches beyond 2^31
    // bags); bf16 as 16 lanes x 16 B, one bag per warp walking runs of up to 8 bags,
    // which keeps it within 64 registers (long bags: the rows dominate)
    case 256:
      if constexpr (BF16) return launch_one<BF16, 16, 1, 8, 8>(a, tab, s);
      else if (static_cast<int64_t>(a.T) * tab.M < (int64_t(1) << 31)) return launch_group<BF16, 8, 2, 4>(a, tab, s);
      else return launch_one<BF16, 8, 2, 4, 1>(a, tab, s);
    case 512: return launch_one<BF16, 32, 1, 8, 1>(a, tab, s);
    case 1024: return launch_one<BF16, 32, 2, 4, 1>(a, tab, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

void preload_gather_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, gather_kernel<false, 1, 1, 1, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<false, 2, 1, 1, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<false, 4, 1, 2, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<false, 8, 1, 4, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<false, 8, 2, 4, 1>);
  cudaFuncGetAttributes(&fa, gather_group_kernel<false, 8, 2, 4>);
  cudaFuncGetAttributes(&fa, gather_kernel<false, 32, 1, 8, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<false, 32, 2, 4, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<true, 1, 1, 1, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<true, 2, 1, 1, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<true, 4, 1, 2, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<true, 8, 1, 4, 4>);
  cudaFuncGetAttributes(&fa, gather_kernel<true, 16, 1, 8, 8>);
  cudaFuncGetAttributes(&fa, gather_kernel<true, 32, 1, 8, 1>);
  cudaFuncGetAttributes(&fa, gather_kernel<true, 32, 2, 4, 1>);
}

cudaError_t launch_gather(const GatherArgs& a, const InvTable& tab, cudaStream_t s) {
  if (a.T < 1 || a.T > kMaxTables || tab.n < 1 || tab.n > kMaxInv) return cudaErrorInvalidValue;
  return a.dtype == 1 ? dispatch<true>(a, tab, s) : dispatch<false>(a, tab, s);
}

}  // namespace sage
