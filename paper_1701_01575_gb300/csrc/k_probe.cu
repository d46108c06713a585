// Measurement only (no counterpart in the paper, which reports no kernel
// throughput).  Instruction issue-rate microbenchmark: warp-instructions per SM per clock
// of one instruction form, measured with eight interleaved dependency chains
// per thread (each step also reads the neighbouring chain, so no chain can be
// folded at compile time) and a 32-warp CTA per SM, so the result is the
// pipe's throughput rather than its latency.  Its figure is the denominator of the kernels'
// roofline (cells per second = SMs x clock x rate x cells per instruction).
#include "dsa_internal.cuh"
#include "dpx.cuh"

#include <algorithm>

namespace dsa {
namespace {

constexpr int PROBE_THREADS = 1024;
constexpr int PROBE_BLOCKS_PER_SM = 1;   // one 32-warp CTA per SM
constexpr int CHAINS = 8;

template <int FORM>
__device__ __forceinline__ uint32_t step(uint32_t x, uint32_t a, uint32_t b) {
  if (FORM == 0) return __viaddmax_s16x2(x, a, b);
  if (FORM == 1) return __vimax_s16x2_relu(x, a);
  if (FORM == 2) return __vimax3_s16x2(x, a, b);
  if (FORM == 3) return x + a;
  if (FORM == 4) {   // inline PTX so the max chain cannot be folded algebraically
    uint32_t r;
    asm volatile("max.s32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(a));
    return r;
  }
  if (FORM == 5) return __vadd2(x, a);
  if (FORM == 6) return (uint32_t)__viaddmax_s32((int)x, (int)a, (int)b);
  if (FORM >= 8 && FORM <= 10) {
    // the empty asm hides the operand's value: a max or saturating chain
    // over known operands could otherwise be folded
    uint32_t y = a;
    asm volatile("" : "+r"(y));
    if (FORM == 8) return __vmaxu4(x, y);
    if (FORM == 9) return __vaddus4(x, y);
    return __vsubus4(x, y);
  }
  return x;
}

template <int FORM>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe(uint32_t a, uint32_t b, int iters,
                                                         uint32_t* sink, long long* cycles) {
  uint32_t v[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) v[c] = threadIdx.x * 7u + c;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) v[c] = step<FORM>(v[c], v[(c + 1) % CHAINS], b + u);
    }
  }
  // pin the results before the closing clock read
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) asm volatile("" ::"r"(v[c]));
  __syncthreads();
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc ^= v[c];
  if (acc == 0x12345678u) sink[threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// The packed local cell update of the inter-sequence kernel, on eight
// independent cells per thread (5 instructions per update).
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_cell(uint32_t neg_o2, uint32_t neg_e2,
                                                              int iters, uint32_t* sink,
                                                              long long* cycles) {
  uint32_t Ho[CHAINS], E[CHAINS], F[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) { Ho[c] = threadIdx.x + c; E[c] = c; F[c] = 3 * c; }
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) {
        const uint32_t old = Ho[c];
        E[c] = __viaddmax_s16x2(E[c], neg_e2, old);
        const uint32_t t = __viaddmax_s16x2(old, 0x00050005u + c, E[c]);
        const uint32_t h = __vimax_s16x2_relu(t, F[c]);
        Ho[c] = __vadd2(h, neg_o2);
        F[c] = __viaddmax_s16x2(F[c], neg_e2, Ho[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) asm volatile("" ::"r"(Ho[c]), "r"(F[c]), "r"(E[c]));
  __syncthreads();
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc ^= Ho[c] ^ F[c];
  if (acc == 0x12345678u) sink[threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// An 8-bit packed local cell update (four cells per register, unsigned
// saturating bytes with a bias, the form of 8-bit striped SIMD
// Smith-Waterman): 10 instructions per update of four cells.
__global__ void __launch_bounds__(PROBE_THREADS) k_probe_cell8(uint32_t o4, uint32_t e4,
                                                               uint32_t bias4, int iters,
                                                               uint32_t* sink, long long* cycles) {
  uint32_t H[CHAINS], E[CHAINS], F[CHAINS], best[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) { H[c] = threadIdx.x + c; E[c] = c; F[c] = 3 * c; best[c] = 0; }
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < 16; ++u) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) {
        uint32_t h = __vaddus4(H[(c + 1) % CHAINS], 0x05030705u + c);   // diagonal + S + bias
        h = __vsubus4(h, bias4);
        h = __vmaxu4(h, E[c]);
        h = __vmaxu4(h, F[c]);
        best[c] = __vmaxu4(best[c], h);
        const uint32_t ho = __vsubus4(h, o4);
        E[c] = __vmaxu4(__vsubus4(E[c], e4), ho);
        F[c] = __vmaxu4(__vsubus4(F[c], e4), ho);
        H[c] = h;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) asm volatile("" ::"r"(H[c]), "r"(F[c]), "r"(E[c]), "r"(best[c]));
  __syncthreads();
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) acc ^= H[c] ^ F[c] ^ best[c];
  if (acc == 0x12345678u) sink[threadIdx.x] = acc;
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
}

// Self-test of the bounded waits: a wait that nothing will ever satisfy must
// give up after `limit_ns`, record DSA_ERR_DEVICE_TIMEOUT in the status word
// and let the kernel return normally.
//   kind 0: an mbarrier whose transaction count is never met (no copy issued);
//   kind 1: a progress flag that no producer ever publishes.
__global__ void k_selftest_wait(int kind, uint64_t limit_ns, uint32_t* flag, int32_t* status) {
  __shared__ uint64_t bar;
  if (kind == 0) {
    if (threadIdx.x == 0) {
      mbar_init(&bar, 1);
      mbar_fence_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) mbar_arrive_expect_tx(&bar, 16);   // no copy will complete it
    __syncthreads();
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (__syncthreads_or(!ok)) {
      if (threadIdx.x == 0) atomicExch(status, DSA_ERR_DEVICE_TIMEOUT);
      return;   // no copy of this CTA is in flight
    }
  } else {
    if (threadIdx.x == 0) {
      const uint64_t t0 = global_ns();
      while (ld_acquire_u32(flag) == 0) {
        if (global_ns() - t0 > limit_ns) {
          atomicExch(status, DSA_ERR_DEVICE_TIMEOUT);
          break;
        }
      }
    }
  }
}

}  // namespace

int run_selftest_wait(dsa_ctx* ctx, int kind, uint64_t limit_ns) {
  if (kind < 0 || kind > 1 || limit_ns > 10000000000ull) {
    set_error("self-test: kind must be 0 or 1 and the limit at most 10 s");
    return DSA_ERR_INVALID_ARG;
  }
  void* flag = nullptr;
  DSA_TRY(ctx->alloc(&flag, sizeof(uint32_t)));
  DSA_CUDA_TRY(cudaMemsetAsync(flag, 0, sizeof(uint32_t), ctx->stream));
  k_selftest_wait<<<1, 64, 0, ctx->stream>>>(kind, limit_ns, static_cast<uint32_t*>(flag),
                                              ctx->d_status);
  ++ctx->launches;
  cudaError_t err = cudaGetLastError();
  ctx->release(flag, sizeof(uint32_t));
  if (err != cudaSuccess) {
    set_error("self-test launch: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  return DSA_OK;
}

int run_issue_probe(dsa_ctx* ctx, int form, double* rate) {
  if (form < 0 || form > 11) {
    set_error("unknown probe form %d", form);
    return DSA_ERR_INVALID_ARG;
  }
  const int blocks = ctx->sm_count * PROBE_BLOCKS_PER_SM;
  const int iters = 4096;
  void* sink = nullptr;
  void* cyc = nullptr;
  DSA_TRY(ctx->alloc(&sink, PROBE_THREADS * sizeof(uint32_t)));
  int rc = ctx->alloc(&cyc, blocks * sizeof(long long));
  if (rc) { ctx->release(sink, PROBE_THREADS * sizeof(uint32_t)); return rc; }
  uint32_t* s = (uint32_t*)sink;
  long long* c = (long long*)cyc;
  const uint32_t a = 0x00030001u, b = 0x00020005u;
  for (int rep = 0; rep < 2; ++rep) {   // first launch warms up
    switch (form) {
      case 0: k_probe<0><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 1: k_probe<1><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 2: k_probe<2><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 3: k_probe<3><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 4: k_probe<4><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 5: k_probe<5><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 6: k_probe<6><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 7: k_probe_cell<<<blocks, PROBE_THREADS, 0, ctx->stream>>>(0xFFF5FFF5u, 0xFFFFFFFFu,
                                                                    iters, s, c); break;
      case 8: k_probe<8><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 9: k_probe<9><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 10: k_probe<10><<<blocks, PROBE_THREADS, 0, ctx->stream>>>(a, b, iters, s, c); break;
      case 11: k_probe_cell8<<<blocks, PROBE_THREADS, 0, ctx->stream>>>(0x0B0B0B0Bu, 0x01010101u,
                                                                     0x04040404u, iters, s, c); break;
    }
  }
  ctx->launches += 2;
  cudaError_t err = cudaGetLastError();
  std::vector<long long> h(blocks);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(h.data(), c, blocks * sizeof(long long), cudaMemcpyDeviceToHost,
                          ctx->stream);
  if (err == cudaSuccess) err = cudaStreamSynchronize(ctx->stream);
  ctx->release(sink, PROBE_THREADS * sizeof(uint32_t));
  ctx->release(cyc, blocks * sizeof(long long));
  if (err != cudaSuccess) {
    set_error("issue probe: %s", cudaGetErrorString(err));
    return DSA_ERR_CUDA;
  }
  std::sort(h.begin(), h.end());
  const double mean = (double)h[h.size() / 2];   // median CTA
  const double instr_per_thread =
      (double)iters * 16 * CHAINS * (form == 7 ? 5 : form == 11 ? 10 : 1);
  const double warp_instr_per_sm =
      instr_per_thread * PROBE_THREADS / 32.0 * PROBE_BLOCKS_PER_SM;
  *rate = warp_instr_per_sm / mean;
  return DSA_OK;
}

}  // namespace dsa
