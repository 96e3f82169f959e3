// Split-precision FP64 matrix products on the 5th-generation tensor cores.
//
// Each FP64 operand row is scaled by a power of two 2^e (|x| < 2^(e-1) over
// the row) and written as k balanced base-128 digits,
//     x = 2^e * sum_{s=1..k} d_s 2^(-7 s),   d_s integer, |d_s| <= 64,
// stored as exact bf16 values.  A product sum_K a b is then
//     2^(ea+eb) * sum_g E_g 2^(-7 g),   E_g = sum_K sum_{i+j=g} d_i^a d_j^b,
// kept for digit orders g = 2 .. k+1 (the remaining orders are below the
// truncation of the digits themselves).  Every digit product is an integer
// <= 2^12 and a group has at most k of them, so E_g is an exact f32 sum while
// K * k * 2^12 < 2^24 (K <= 640 for k <= 6).  Each group accumulates in its own
// TMEM accumulator (tcgen05.mma kind::f16, bf16 x bf16 -> f32); the epilogue
// recombines the exact integers W = sum_g E_g 2^(7 (k+1-g)) in int64, so the
// recombination is exact and the result carries about 7k significant bits
// relative to 2^(ea+eb).
//
// Kernel structure (one CTA = one 128 x NT output tile, 4 warps):
//   thread 0 streams A and B digit tiles with 1-D bulk copies (TMA) into a
//   two-stage shared-memory ring guarded by mbarriers and issues the
//   k(k+1)/2 MMAs per K = 16 step; all four warps then read the k
//   accumulators from TMEM (each warp its 32 lanes) and run the epilogue.
#include <cuda_bf16.h>

#include <algorithm>
#include <vector>

#include "umma.cuh"

namespace oz {

constexpr int TM = 128;     // A-tile rows (MMA M)
constexpr int TK = 32;      // K per tile
constexpr int KMAX = 640;   // exact group sums: K * k * 2^12 < 2^24 for k <= 6
constexpr int NSTAGE = 2;

// element offset of (r, c) in a [rows x 32] K-major core-matrix tile
__host__ __device__ __forceinline__ int tile_off(int r, int c) {
  return ((r >> 3) * 4 + (c >> 3)) * 64 + (r & 7) * 8 + (c & 7);
}

struct Problem {
  const __nv_bfloat16 *A;  // [mtiles][ktiles][k][TM*TK]
  const __nv_bfloat16 *B;  // [ntiles][ktiles][k][NT*TK]
  const int16_t *ea;       // per A row
  const int16_t *eb;       // per B row (output column)
  int mtiles, ntiles, ktiles;
  int M, N;
  double *C;               // row-major output (plain store)
  int64_t ldc;
  int64_t cta_base;        // first CTA of this problem
};

// One warp per operand row: exponent, then k balanced digits per element.
// Element (r, c) of the logical R x K operand is X[r * rs + c * cs].
template <int KS>
__global__ void k_slice(const double *__restrict__ X, int64_t rs, int64_t cs, int R, int K,
                        int rows_pt, int ktiles, int nrows_padded, __nv_bfloat16 *out,
                        int16_t *eout) {
  const int r = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= nrows_padded) return;
  const int Kp = ktiles * TK;
  long long mbits = 0;
  if (r < R)
    for (int c = lane; c < K; c += 32) {
      const long long b = __double_as_longlong(X[(int64_t)r * rs + (int64_t)c * cs]) &
                          0x7FFFFFFFFFFFFFFFll;
      mbits = max(mbits, b);
    }
  for (int o = 16; o; o >>= 1) mbits = max(mbits, __shfl_xor_sync(0xffffffffu, mbits, o));
  int e = -1000;
  if (mbits != 0) {
    const int ef = (int)(mbits >> 52);
    e = (ef == 0 ? -1022 : ef - 1023) + 2;  // |x| < 2^(e-1)
  }
  if (lane == 0) eout[r] = (int16_t)max(-30000, e);
  const int rt = r / rows_pt, rr = r - rt * rows_pt;
  for (int c = lane; c < Kp; c += 32) {
    double x = 0.0;
    if (r < R && c < K && e > -1000) x = X[(int64_t)r * rs + (int64_t)c * cs];
    long long Xi = (e > -1000) ? __double2ll_rn(ldexp(x, 7 * KS - e)) : 0ll;
    int d[KS];
#pragma unroll
    for (int s = KS - 1; s > 0; --s) {
      const int dd = (int)(((Xi + 64) & 127) - 64);
      d[s] = dd;
      Xi = (Xi - dd) >> 7;
    }
    d[0] = (int)Xi;
    const int kt = c / TK, cc = c - kt * TK;
    __nv_bfloat16 *base = out + ((int64_t)(rt * ktiles + kt) * KS) * rows_pt * TK;
#pragma unroll
    for (int s = 0; s < KS; ++s)
      base[(int64_t)s * rows_pt * TK + tile_off(rr, cc)] = __int2bfloat16_rn(d[s]);
  }
}

__host__ __device__ constexpr uint32_t tmem_cols(int ks, int nt) {
  return (uint32_t)(ks * nt <= 32 ? 32 : ks * nt <= 64 ? 64 : ks * nt <= 128 ? 128
                    : ks * nt <= 256 ? 256 : 512);
}

template <int NT, int KS>
__global__ void __launch_bounds__(128, 1) k_gemm(const Problem *__restrict__ probs, int nprob,
                                                 unsigned *err) {
  extern __shared__ __align__(1024) uint8_t smem[];
  constexpr int A_BYTES = KS * TM * TK * 2;
  constexpr int B_BYTES = KS * NT * TK * 2;
  constexpr int STAGE = A_BYTES + B_BYTES;
  constexpr uint32_t TCOLS = tmem_cols(KS, NT);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + NSTAGE * STAGE);
  uint64_t *empty = full + NSTAGE;
  uint64_t *done = empty + NSTAGE;
  uint32_t *tslot = reinterpret_cast<uint32_t *>(done + 1);

  // problem and tile of this CTA
  int lo = 0, hi = nprob - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (probs[mid].cta_base <= (int64_t)blockIdx.x) lo = mid; else hi = mid - 1;
  }
  const Problem &P = probs[lo];
  const int local = (int)((int64_t)blockIdx.x - P.cta_base);
  const int mt = local / P.ntiles, nt = local - mt * P.ntiles;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NSTAGE; ++s) {
      umma::mbar_init(&full[s], 1);
      umma::mbar_init(&empty[s], 1);
    }
    umma::mbar_init(done, 1);
    umma::fence_barrier_init();
  }
  if (warp == 0) {
    umma::tmem_alloc(tslot, TCOLS);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tbase = *tslot;

  if (threadIdx.x == 0) {
    const __nv_bfloat16 *Ab = P.A + (int64_t)mt * P.ktiles * KS * TM * TK;
    const __nv_bfloat16 *Bb = P.B + (int64_t)nt * P.ktiles * KS * NT * TK;
    constexpr uint32_t idesc = umma::idesc_bf16_f32(TM, NT);
    auto load = [&](int s, int kt) {
      umma::mbar_arrive_expect_tx(&full[s], STAGE);
      umma::bulk_g2s(smem + s * STAGE, Ab + (int64_t)kt * KS * TM * TK, A_BYTES, &full[s]);
      umma::bulk_g2s(smem + s * STAGE + A_BYTES, Bb + (int64_t)kt * KS * NT * TK, B_BYTES,
                     &full[s]);
    };
    for (int s = 0; s < NSTAGE && s < P.ktiles; ++s) load(s, s);
    bool ok = true;
    for (int kt = 0; kt < P.ktiles; ++kt) {
      const int s = kt % NSTAGE;
      const uint32_t ph = (uint32_t)(kt / NSTAGE) & 1u;
      if (!umma::mbar_wait(&full[s], ph, err)) { ok = false; break; }
      umma::fence_after_sync();
      const uint32_t a0 = umma::smem_u32(smem + s * STAGE), b0 = a0 + A_BYTES;
#pragma unroll
      for (int j = 0; j < TK / 16; ++j)
#pragma unroll
        for (int g = 0; g < KS; ++g)
#pragma unroll
          for (int i = 0; i <= g; ++i) {
            const uint64_t ad = umma::smem_desc(a0 + i * TM * TK * 2 + j * 256, 128, 512);
            const uint64_t bd = umma::smem_desc(b0 + (g - i) * NT * TK * 2 + j * 256, 128, 512);
            umma::mma_bf16(tbase + g * NT, ad, bd, idesc, (kt | j | i) ? 1u : 0u);
          }
      umma::mma_commit(&empty[s]);
      if (kt + NSTAGE < P.ktiles) {
        if (!umma::mbar_wait(&empty[s], ph, err)) { ok = false; break; }
        load(s, kt + NSTAGE);
      }
    }
    if (ok) {
      umma::mma_commit(done);
    } else {
      asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(done)) : "memory");
    }
  }
  __syncwarp();
  const bool ready = umma::mbar_wait(done, 0, err);
  umma::fence_after_sync();
  // epilogue: warp w owns TMEM lanes (rows) 32w .. 32w+31
  const int row = warp * 32 + lane;
  const int m = mt * TM + row;
  const int ea = (m < P.M) ? P.ea[m] : 0;
  for (int c0 = 0; c0 < NT; c0 += 32) {
    long long W[32];
#pragma unroll
    for (int i = 0; i < 32; ++i) W[i] = 0;
#pragma unroll
    for (int g = 0; g < KS; ++g) {
      float v[32];
      umma::tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(g * NT + c0), v);
      const long long sc = 1ll << (7 * (KS - 1 - g));
#pragma unroll
      for (int i = 0; i < 32; ++i) W[i] += (long long)__float2int_rn(v[i]) * sc;
    }
    if (ready && m < P.M) {
#pragma unroll
      for (int i = 0; i < 32; ++i) {
        const int n = nt * NT + c0 + i;
        if (n < P.N) P.C[(int64_t)m * P.ldc + n] = ldexp((double)W[i], ea + P.eb[n] - 7 * (KS + 1));
      }
    }
  }
  umma::fence_before_sync();
  __syncthreads();
  if (warp == 0) umma::tmem_dealloc(tbase, TCOLS);
}

template <int NT, int KS>
size_t gemm_smem() {
  constexpr int STAGE = KS * (TM + NT) * TK * 2;
  const size_t need = (size_t)NSTAGE * STAGE + 64;
  // keep the CTAs an SM can hold within TMEM (512 columns), so tcgen05.alloc never waits
  const int limit = 512 / (int)tmem_cols(KS, NT);
  const size_t floor_bytes = (size_t)(233472 / (limit + 1)) + 1024;
  return std::max(need, floor_bytes);
}

template <int NT, int KS>
cudaError_t launch_gemm(const Problem *d_probs, int nprob, int64_t nctas, unsigned *err,
                        cudaStream_t st) {
  const size_t sm = gemm_smem<NT, KS>();
  cudaError_t e = cudaFuncSetAttribute(k_gemm<NT, KS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)sm);
  if (e != cudaSuccess) return e;
  k_gemm<NT, KS><<<(unsigned)nctas, 128, sm, st>>>(d_probs, nprob, err);
  return cudaGetLastError();
}

template <int KS>
cudaError_t launch_slice(const double *X, int64_t rs, int64_t cs, int R, int K, int rows_pt,
                         int ktiles, int nrows_padded, __nv_bfloat16 *out, int16_t *eout,
                         cudaStream_t st) {
  const int64_t threads = (int64_t)nrows_padded * 32;
  k_slice<KS><<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(X, rs, cs, R, K, rows_pt, ktiles,
                                                                nrows_padded, out, eout);
  return cudaGetLastError();
}

template <int KS>
hfx_status selftest(int M, int N, int K, const double *A, const double *B, double *C) {
  constexpr int NT = 64;
  const int mtiles = (M + TM - 1) / TM, ntiles = (N + NT - 1) / NT, ktiles = (K + TK - 1) / TK;
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  __nv_bfloat16 *sA = nullptr, *sB = nullptr;
  int16_t *eA = nullptr, *eB = nullptr;
  unsigned *dErr = nullptr;
  Problem *dP = nullptr;
  hfx_status status = HFX_E_CUDA;
  const size_t nsA = (size_t)mtiles * ktiles * KS * TM * TK;
  const size_t nsB = (size_t)ntiles * ktiles * KS * NT * TK;
  do {
    if (cudaMalloc(&dA, sizeof(double) * M * K) || cudaMalloc(&dB, sizeof(double) * K * N) ||
        cudaMalloc(&dC, sizeof(double) * M * N) || cudaMalloc(&sA, 2 * nsA) ||
        cudaMalloc(&sB, 2 * nsB) || cudaMalloc(&eA, 2 * mtiles * TM) ||
        cudaMalloc(&eB, 2 * ntiles * NT) || cudaMalloc(&dErr, sizeof(unsigned)) ||
        cudaMalloc(&dP, sizeof(Problem))) {
      status = HFX_E_NOMEM;
      break;
    }
    if (cudaMemcpy(dA, A, sizeof(double) * M * K, cudaMemcpyHostToDevice) ||
        cudaMemcpy(dB, B, sizeof(double) * K * N, cudaMemcpyHostToDevice) ||
        cudaMemset(dErr, 0, sizeof(unsigned)))
      break;
    // A rows: r = m, element (m, k) at m*K + k; B "rows" are its columns n: (n, k) at k*N + n
    if (launch_slice<KS>(dA, K, 1, M, K, TM, ktiles, mtiles * TM, sA, eA, 0) ||
        launch_slice<KS>(dB, 1, N, N, K, NT, ktiles, ntiles * NT, sB, eB, 0))
      break;
    Problem p{};
    p.A = sA; p.B = sB; p.ea = eA; p.eb = eB;
    p.mtiles = mtiles; p.ntiles = ntiles; p.ktiles = ktiles;
    p.M = M; p.N = N; p.C = dC; p.ldc = N; p.cta_base = 0;
    if (cudaMemcpy(dP, &p, sizeof(Problem), cudaMemcpyHostToDevice)) break;
    if (launch_gemm<NT, KS>(dP, 1, (int64_t)mtiles * ntiles, dErr, 0)) break;
    unsigned herr = 0;
    if (cudaMemcpy(&herr, dErr, sizeof(unsigned), cudaMemcpyDeviceToHost)) break;
    if (herr) { status = herr & HFX_DEV_ERR_TIMEOUT ? HFX_E_TIMEOUT : HFX_E_CUDA; break; }
    if (cudaMemcpy(C, dC, sizeof(double) * M * N, cudaMemcpyDeviceToHost)) break;
    status = HFX_OK;
  } while (0);
  cudaFree(dA); cudaFree(dB); cudaFree(dC); cudaFree(sA); cudaFree(sB);
  cudaFree(eA); cudaFree(eB); cudaFree(dErr); cudaFree(dP);
  return status;
}

}  // namespace oz

extern "C" hfx_status hfx_selftest_ozaki(int32_t M, int32_t N, int32_t K, const double *A,
                                         const double *B, double *C, int32_t nslices) {
  if (!A || !B || !C || M < 1 || N < 1 || K < 1 || K > oz::KMAX) return HFX_E_ARG;
  switch (nslices) {
    case 1: return oz::selftest<1>(M, N, K, A, B, C);
    case 2: return oz::selftest<2>(M, N, K, A, B, C);
    case 3: return oz::selftest<3>(M, N, K, A, B, C);
    case 4: return oz::selftest<4>(M, N, K, A, B, C);
    case 5: return oz::selftest<5>(M, N, K, A, B, C);
    case 6: return oz::selftest<6>(M, N, K, A, B, C);
    default: return HFX_E_ARG;
  }
}

namespace oz {

// One thread waits, with the kernels' bounded wait, on an mbarrier nothing
// arrives at; the expiry is recorded in *err and the kernel returns.
__global__ void k_wait_nothing(long long limit, unsigned *err, long long *waited) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x != 0) return;
  umma::mbar_init(&bar, 1);
  umma::fence_barrier_init();
  const long long t0 = clock64();
  umma::mbar_wait(&bar, 0, err, limit);
  *waited = clock64() - t0;
}

}  // namespace oz

extern "C" hfx_status hfx_selftest_timeout(int64_t limit_cycles, int64_t *waited_cycles) {
  if (limit_cycles < 1 || limit_cycles > 2000000000ll) return HFX_E_ARG;
  unsigned *d_err = nullptr;
  long long *d_w = nullptr;
  if (cudaMalloc((void **)&d_err, sizeof(unsigned)) != cudaSuccess) return HFX_E_CUDA;
  if (cudaMalloc((void **)&d_w, sizeof(long long)) != cudaSuccess) {
    cudaFree(d_err);
    return HFX_E_CUDA;
  }
  hfx_status st = HFX_OK;
  unsigned herr = 0;
  long long hw = 0;
  if (cudaMemset(d_err, 0, sizeof(unsigned)) != cudaSuccess) st = HFX_E_CUDA;
  if (st == HFX_OK) {
    oz::k_wait_nothing<<<1, 32>>>(limit_cycles, d_err, d_w);
    if (cudaDeviceSynchronize() != cudaSuccess ||
        cudaMemcpy(&herr, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(&hw, d_w, sizeof(long long), cudaMemcpyDeviceToHost) != cudaSuccess)
      st = HFX_E_CUDA;
  }
  cudaFree(d_err);
  cudaFree(d_w);
  if (st != HFX_OK) return st;
  if (waited_cycles) *waited_cycles = hw;
  return (herr & HFX_DEV_ERR_TIMEOUT) ? HFX_E_TIMEOUT : HFX_OK;
}
