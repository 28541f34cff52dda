// CUDA-core kernels of the MLPs: the fp32 GEMM (fp32 functions), the thin
// bottom layer 0 (K = number of dense features) and the sigmoid head (N = 1).
//
// Every output element is one fp32 FMA chain over k = 0..K-1 followed by the
// bias, so its value does not depend on M, on the tile it falls in or on the
// other rows of the batch.
#include "kernels.h"

namespace sage {
namespace {

// ---------------------------------------------------------------- fp32 GEMM
// C[M,N] = act(A[M,K] W[N,K]^T + b).  Tile BM x BN x BK, 256 threads, each
// thread owns a TM x TN block split in two halves of 4 rows / 4 columns that are
// BM/2 (BN/2) apart, so that shared-memory float4 reads are conflict-free.
template <int BM, int BN, int BK>
__global__ void __launch_bounds__(256, 2) sgemm_nt_kernel(int M, int N, int K, const float* __restrict__ A, int lda,
                                                       const float* __restrict__ W, const float* __restrict__ bias,
                                                       int relu, float* __restrict__ C, int ldc) {
  constexpr int TM = BM / 16, TN = BN / 16;  // 16 x 16 threads
  constexpr int TX = 16;
  constexpr int NH = TN / 4;                 // column groups of 4 per thread
  static_assert(TM == 8 && (TN == 8 || TN == 4), "tile shape");
  __shared__ __align__(16) float As[2][BK][BM];
  __shared__ __align__(16) float Ws[2][BK][BN];

  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;

  // global -> shared staging: each thread moves (BM*BK/4)/256 float4 of A and of W
  constexpr int A_V4 = BM * BK / 4 / 256;
  constexpr int W_V4 = BN * BK / 4 / 256;
  float4 ra[A_V4 > 0 ? A_V4 : 1], rw[W_V4 > 0 ? W_V4 : 1];

  auto load_tiles = [&](int k0) {
#pragma unroll
    for (int q = 0; q < A_V4; ++q) {
      const int v = tid + q * 256;
      const int row = v / (BK / 4), kq = (v % (BK / 4)) * 4;
      const int gm = m0 + row, gk = k0 + kq;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gm < M) {
        if (gk + 3 < K) {
          x = *reinterpret_cast<const float4*>(A + static_cast<size_t>(gm) * lda + gk);
        } else {
          const float* p = A + static_cast<size_t>(gm) * lda;
          x.x = gk < K ? p[gk] : 0.f;
          x.y = gk + 1 < K ? p[gk + 1] : 0.f;
          x.z = gk + 2 < K ? p[gk + 2] : 0.f;
          x.w = gk + 3 < K ? p[gk + 3] : 0.f;
        }
      }
      ra[q] = x;
    }
#pragma unroll
    for (int q = 0; q < W_V4; ++q) {
      const int v = tid + q * 256;
      const int row = v / (BK / 4), kq = (v % (BK / 4)) * 4;
      const int gn = n0 + row, gk = k0 + kq;
      float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gn < N) {
        if (gk + 3 < K) {
          x = *reinterpret_cast<const float4*>(W + static_cast<size_t>(gn) * K + gk);
        } else {
          const float* p = W + static_cast<size_t>(gn) * K;
          x.x = gk < K ? p[gk] : 0.f;
          x.y = gk + 1 < K ? p[gk + 1] : 0.f;
          x.z = gk + 2 < K ? p[gk + 2] : 0.f;
          x.w = gk + 3 < K ? p[gk + 3] : 0.f;
        }
      }
      rw[q] = x;
    }
  };
  auto store_tiles = [&](int buf) {
#pragma unroll
    for (int q = 0; q < A_V4; ++q) {
      const int v = tid + q * 256;
      const int row = v / (BK / 4), kq = (v % (BK / 4)) * 4;
      As[buf][kq + 0][row] = ra[q].x;
      As[buf][kq + 1][row] = ra[q].y;
      As[buf][kq + 2][row] = ra[q].z;
      As[buf][kq + 3][row] = ra[q].w;
    }
#pragma unroll
    for (int q = 0; q < W_V4; ++q) {
      const int v = tid + q * 256;
      const int row = v / (BK / 4), kq = (v % (BK / 4)) * 4;
      Ws[buf][kq + 0][row] = rw[q].x;
      Ws[buf][kq + 1][row] = rw[q].y;
      Ws[buf][kq + 2][row] = rw[q].z;
      Ws[buf][kq + 3][row] = rw[q].w;
    }
  };

  float acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;

  const int ktiles = (K + BK - 1) / BK;
  load_tiles(0);
  store_tiles(0);
  __syncthreads();
  for (int kt = 0; kt < ktiles; ++kt) {
    const int buf = kt & 1;
    if (kt + 1 < ktiles) load_tiles((kt + 1) * BK);
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      float a[TM], w[TN];
      const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][BM / 2 + ty * 4]);
      a[0] = a0.x; a[1] = a0.y; a[2] = a0.z; a[3] = a0.w;
      a[4] = a1.x; a[5] = a1.y; a[6] = a1.z; a[7] = a1.w;
#pragma unroll
      for (int h = 0; h < NH; ++h) {
        const float4 wv = *reinterpret_cast<const float4*>(&Ws[buf][kk][h * (BN / 2) + tx * 4]);
        w[4 * h + 0] = wv.x; w[4 * h + 1] = wv.y; w[4 * h + 2] = wv.z; w[4 * h + 3] = wv.w;
      }
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fmaf(a[i], w[j], acc[i][j]);
    }
    if (kt + 1 < ktiles) store_tiles(buf ^ 1);
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + (i < 4 ? ty * 4 + i : BM / 2 + ty * 4 + (i - 4));
    if (gm >= M) continue;
#pragma unroll
    for (int h = 0; h < NH; ++h) {
      const int gn = n0 + h * (BN / 2) + tx * 4;
      if (gn >= N) continue;
      float o[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        float v = acc[i][h * 4 + j] + (gn + j < N ? bias[gn + j] : 0.f);
        o[j] = relu ? fmaxf(v, 0.f) : v;
      }
      float* dst = C + static_cast<size_t>(gm) * ldc + gn;
      if (gn + 3 < N) {
        *reinterpret_cast<float4*>(dst) = make_float4(o[0], o[1], o[2], o[3]);
      } else {
        for (int j = 0; j < 4 && gn + j < N; ++j) dst[j] = o[j];
      }
    }
  }
}

// ---------------------------------------------------------------- bottom layer 0
// One warp per batch row: the row's K dense features (K <= 64) are read from its
// invocation; W0 and b0 sit in shared memory as fp32; lane l computes outputs
// l, l+32, ... (coalesced stores).
template <bool BF16>
__global__ void __launch_bounds__(256) bottom0_kernel(const __grid_constant__ InvTable tab, int K, int N,
                                                      const void* __restrict__ Wv, const float* __restrict__ bias,
                                                      void* __restrict__ y, int ldy, float* __restrict__ y_lo) {
  extern __shared__ float sm[];  // [N*K] weights then [N] bias
  float* sW = sm;
  float* sb = sm + static_cast<size_t>(N) * K;
  for (int e = threadIdx.x; e < N * K; e += blockDim.x) {
    if (BF16) {
      const uint16_t u = reinterpret_cast<const uint16_t*>(Wv)[e];
      sW[e] = __uint_as_float(static_cast<uint32_t>(u) << 16);
    } else {
      sW[e] = reinterpret_cast<const float*>(Wv)[e];
    }
  }
  for (int e = threadIdx.x; e < N; e += blockDim.x) sb[e] = bias[e];
  __syncthreads();

  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < tab.M; r += warps) {
    const int i = tab.n == 1 ? 0 : find_inv(tab, r);
    const float* x = tab.d[i].dense + static_cast<size_t>(r - tab.d[i].row_base) * K;
    const float xl = lane < K ? x[lane] : 0.f;
    const float xh = lane + 32 < K ? x[lane + 32] : 0.f;
    for (int j0 = 0; j0 < N; j0 += 32) {
      const int j = j0 + lane;
      const int jr = j < N ? j : N - 1;
      float s = 0.f;
      const float* w = sW + static_cast<size_t>(jr) * K;
      for (int k = 0; k < K; ++k) {
        const float xk = __shfl_sync(0xffffffffu, k < 32 ? xl : xh, k & 31);
        s = fmaf(xk, w[k], s);
      }
      if (j >= N) continue;
      s = fmaxf(s + sb[j], 0.f);
      const size_t o = static_cast<size_t>(r) * ldy + j;
      if (BF16) {
        reinterpret_cast<__nv_bfloat16*>(y)[o] = __float2bfloat16_rn(s);
      } else if (y_lo) {
        const float h = to_tf32_rna(s);
        reinterpret_cast<float*>(y)[o] = h;
        y_lo[o] = s - h;
      } else {
        reinterpret_cast<float*>(y)[o] = s;
      }
    }
  }
}

// Bottom layer 0 for thin inputs (K <= 16): a block walks groups of 32 rows
// (grid-stride) and computes all N outputs of each; each thread keeps one or two
// output columns' weights in registers for the whole walk, and the group's dense
// features sit in shared memory (broadcast reads).  Stores are coalesced along the
// output row.  Same per-output order as above (k = 0..K-1 FMA chain, then the bias).
template <bool BF16>
__global__ void __launch_bounds__(256) bottom0_thin_kernel(const __grid_constant__ InvTable tab, int K, int N,
                                                           const void* __restrict__ Wv,
                                                           const float* __restrict__ bias, void* __restrict__ y,
                                                           int ldy, float* __restrict__ y_lo) {
  constexpr int R = 32, KM = 16;
  __shared__ __align__(16) float sx[R][KM];  // dense rows, zero-padded to KM
  __shared__ const float* srow[R];
  // the group's dense rows into shared memory (callers sync before reuse)
  auto stage = [&](int r0) {
    if (threadIdx.x < R) {
      const int r = r0 + threadIdx.x;
      const float* p = nullptr;
      if (r < tab.M) {
        const int i = tab.n == 1 ? 0 : find_inv(tab, r);
        p = tab.d[i].dense + static_cast<size_t>(r - tab.d[i].row_base) * K;
      }
      srow[threadIdx.x] = p;
    }
    __syncthreads();
    for (int e = threadIdx.x; e < R * KM; e += blockDim.x) {
      const int rr = e / KM, k = e % KM;
      sx[rr][k] = (srow[rr] && k < K) ? srow[rr][k] : 0.f;
    }
    __syncthreads();
  };
  auto load_w = [&](int j, float (&w)[KM]) {
#pragma unroll
    for (int k = 0; k < KM; ++k) {
      if (k < K) {
        if (BF16) {
          const uint16_t u = reinterpret_cast<const uint16_t*>(Wv)[static_cast<size_t>(j) * K + k];
          w[k] = __uint_as_float(static_cast<uint32_t>(u) << 16);
        } else {
          w[k] = reinterpret_cast<const float*>(Wv)[static_cast<size_t>(j) * K + k];
        }
      } else {
        w[k] = 0.f;
      }
    }
  };
  // k order 0..KM-1; the padded terms (k >= K) add 0 * 0 and leave s unchanged
  auto dot = [&](const float4 (&x)[KM / 4], const float (&w)[KM], float b) {
    float s = 0.f;
#pragma unroll
    for (int q = 0; q < KM / 4; ++q) {
      s = fmaf(x[q].x, w[4 * q], s);
      s = fmaf(x[q].y, w[4 * q + 1], s);
      s = fmaf(x[q].z, w[4 * q + 2], s);
      s = fmaf(x[q].w, w[4 * q + 3], s);
    }
    return fmaxf(s + b, 0.f);
  };
  auto store1 = [&](size_t o, float v) {
    if (BF16) {
      reinterpret_cast<__nv_bfloat16*>(y)[o] = __float2bfloat16_rn(v);
    } else if (y_lo) {
      const float h = to_tf32_rna(v);
      reinterpret_cast<float*>(y)[o] = h;
      y_lo[o] = v - h;
    } else {
      reinterpret_cast<float*>(y)[o] = v;
    }
  };
  // two adjacent columns per thread (one 8-byte / bf16-pair store per row and plane)
  // when the layout allows it
  const bool pairs = (N % 2 == 0) && (ldy % 2 == 0) && !(reinterpret_cast<uintptr_t>(y) & 7) &&
                     !(reinterpret_cast<uintptr_t>(y_lo) & 7);
  const int per = pairs ? 2 : 1;
  if (N <= per * static_cast<int>(blockDim.x)) {
    // every column of the layer has its thread: weights stay in registers for the walk
    const int j = per * static_cast<int>(threadIdx.x);
    const bool act = j < N;
    float w0[KM], w1[KM];
    float b0 = 0.f, b1 = 0.f;
    if (act) {
      load_w(j, w0);
      b0 = bias[j];
      if (pairs) {
        load_w(j + 1, w1);
        b1 = bias[j + 1];
      }
    }
    for (int r0 = blockIdx.x * R; r0 < tab.M; r0 += gridDim.x * R) {
      stage(r0);
      const int nrows = min(R, tab.M - r0);
      if (act) {
        for (int rr = 0; rr < nrows; ++rr) {
          float4 x[KM / 4];
#pragma unroll
          for (int q = 0; q < KM / 4; ++q) x[q] = reinterpret_cast<const float4*>(&sx[rr][0])[q];  // broadcasts
          const size_t o = static_cast<size_t>(r0 + rr) * ldy + j;
          const float s0 = dot(x, w0, b0);
          if (pairs) {
            const float s1 = dot(x, w1, b1);
            if (BF16) {
              *reinterpret_cast<uint32_t*>(reinterpret_cast<__nv_bfloat16*>(y) + o) = pack_bf16x2(s0, s1);
            } else if (y_lo) {
              const float h0 = to_tf32_rna(s0), h1 = to_tf32_rna(s1);
              *reinterpret_cast<float2*>(reinterpret_cast<float*>(y) + o) = make_float2(h0, h1);
              *reinterpret_cast<float2*>(y_lo + o) = make_float2(s0 - h0, s1 - h1);
            } else {
              *reinterpret_cast<float2*>(reinterpret_cast<float*>(y) + o) = make_float2(s0, s1);
            }
          } else {
            store1(o, s0);
          }
        }
      }
      __syncthreads();  // before the next group overwrites sx
    }
    return;
  }
  // wider layers: columns in strides of the block, weights reloaded per group
  for (int r0 = blockIdx.x * R; r0 < tab.M; r0 += gridDim.x * R) {
    stage(r0);
    const int nrows = min(R, tab.M - r0);
    for (int j = threadIdx.x; j < N; j += blockDim.x) {
      float w[KM];
      load_w(j, w);
      const float bj = bias[j];
      for (int rr = 0; rr < nrows; ++rr) {
        float4 x[KM / 4];
#pragma unroll
        for (int q = 0; q < KM / 4; ++q) x[q] = reinterpret_cast<const float4*>(&sx[rr][0])[q];
        store1(static_cast<size_t>(r0 + rr) * ldy + j, dot(x, w, bj));
      }
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- head
// One warp per batch row: z = h . w + c in the fixed head order (a 32-column
// chunk per load, lane j holding column k0 + j, summed by xor shuffles), out =
// 1 / (1 + exp(-z)) written to the row's invocation.
template <bool BF16>
__global__ void __launch_bounds__(256) head_kernel(const __grid_constant__ InvTable tab, int K,
                                                  const void* __restrict__ h, int ldh, const void* __restrict__ w,
                                                  const float* __restrict__ c, const float* __restrict__ h_lo) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  auto chunk = [&](int r, int k0) {
    const int k = k0 + lane;
    float p = 0.f;
    if (k < K) {
      float hv, wv;
      if (BF16) {
        hv = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(h)[static_cast<size_t>(r) * ldh + k]);
        wv = __bfloat162float(reinterpret_cast<const __nv_bfloat16*>(w)[k]);
      } else {
        const size_t o = static_cast<size_t>(r) * ldh + k;
        // hi + lo planes: the sum is the fp32 value exactly (lo is the exact residual)
        hv = h_lo ? __fadd_rn(reinterpret_cast<const float*>(h)[o], h_lo[o]) : reinterpret_cast<const float*>(h)[o];
        wv = reinterpret_cast<const float*>(w)[k];
      }
      p = __fmul_rn(hv, wv);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) p = __fadd_rn(p, __shfl_xor_sync(0xffffffffu, p, o));
    return p;
  };
  for (int r = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; r < tab.M; r += warps) {
    float z = 0.f;
    for (int k0 = 0; k0 < K; k0 += 64) {
      const float g = __fadd_rn(chunk(r, k0), chunk(r, k0 + 32));
      z = k0 == 0 ? g : __fadd_rn(z, g);
    }
    if (lane == 0) {
      const int i = tab.n == 1 ? 0 : find_inv(tab, r);
      tab.d[i].out[r - tab.d[i].row_base] = head_sigmoid(__fadd_rn(z, c[0]));
    }
  }
}

int sms() { return device_sms(); }

}  // namespace

void preload_simt_kernels() {
  cudaFuncAttributes fa;
  cudaFuncGetAttributes(&fa, sgemm_nt_kernel<128, 64, 16>);
  cudaFuncGetAttributes(&fa, sgemm_nt_kernel<128, 128, 16>);
  cudaFuncGetAttributes(&fa, bottom0_kernel<false>);
  cudaFuncGetAttributes(&fa, bottom0_kernel<true>);
  cudaFuncGetAttributes(&fa, bottom0_thin_kernel<false>);
  cudaFuncGetAttributes(&fa, bottom0_thin_kernel<true>);
  cudaFuncGetAttributes(&fa, head_kernel<false>);
  cudaFuncGetAttributes(&fa, head_kernel<true>);
}

cudaError_t launch_linear_f32(int M, int N, int K, const float* x, int ldx, const float* W, const float* bias,
                              int relu, float* y, int ldy, cudaStream_t s) {
  if (M <= 0) return cudaSuccess;
  if ((ldx & 3) || (K & 3) || (ldy & 3) || (N & 3)) return cudaErrorInvalidValue;
  // 128x64 tiles when 128x128 would leave most SMs idle
  const int tiles128 = ((M + 127) / 128) * ((N + 127) / 128);
  if (N <= 64 || tiles128 < 2 * sms()) {
    dim3 grid((N + 63) / 64, (M + 127) / 128);
    sgemm_nt_kernel<128, 64, 16><<<grid, 256, 0, s>>>(M, N, K, x, ldx, W, bias, relu, y, ldy);
  } else {
    dim3 grid((N + 127) / 128, (M + 127) / 128);
    sgemm_nt_kernel<128, 128, 16><<<grid, 256, 0, s>>>(M, N, K, x, ldx, W, bias, relu, y, ldy);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_bottom0(int dtype, const InvTable& tab, int K, int N, const void* W, const float* bias,
                           void* y, int ldy, cudaStream_t s, float* y_lo) {
  if (tab.M <= 0) return cudaSuccess;
  if (K < 1 || K > 64) return cudaErrorInvalidValue;
  if (K <= 16) {
    // groups of 32 rows, walked by one wave of blocks (4 per SM at <= 64 registers)
    const int blocks = std::min((tab.M + 31) / 32, sms() * 4);
    if (dtype == 1) bottom0_thin_kernel<true><<<blocks, 256, 0, s>>>(tab, K, N, W, bias, y, ldy, nullptr);
    else bottom0_thin_kernel<false><<<blocks, 256, 0, s>>>(tab, K, N, W, bias, y, ldy, y_lo);
    count_launch();
    return cudaGetLastError();
  }
  const size_t smem = (static_cast<size_t>(N) * K + N) * sizeof(float);
  if (smem > 200 * 1024) return cudaErrorInvalidValue;
  int blocks = (tab.M + 7) / 8;
  const int cap = sms() * 4;
  if (blocks > cap) blocks = cap;
  if (dtype == 1) {
    cudaFuncSetAttribute(bottom0_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    bottom0_kernel<true><<<blocks, 256, smem, s>>>(tab, K, N, W, bias, y, ldy, nullptr);
  } else {
    cudaFuncSetAttribute(bottom0_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
    bottom0_kernel<false><<<blocks, 256, smem, s>>>(tab, K, N, W, bias, y, ldy, y_lo);
  }
  count_launch();
  return cudaGetLastError();
}

cudaError_t launch_head(int dtype, const InvTable& tab, int K, const void* h, int ldh, const void* w,
                        const float* c, cudaStream_t s, const float* h_lo) {
  if (tab.M <= 0) return cudaSuccess;
  int blocks = (tab.M + 7) / 8;
  const int cap = sms() * 8;
  if (blocks > cap) blocks = cap;
  if (dtype == 1) {
    head_kernel<true><<<blocks, 256, 0, s>>>(tab, K, h, ldh, w, c, nullptr);
  } else {
    head_kernel<false><<<blocks, 256, 0, s>>>(tab, K, h, ldh, w, c, h_lo);
  }
  count_launch();
  return cudaGetLastError();
}

}  // namespace sage
