// train_tc.cu -- (a6) the three GEMM shapes of a training step of the residual
// network (Sec. VI: MSE loss, Adam) on the tcgen05 tensor cores:
//   forward         Z_{l+1} = W_l A_l + b_l,  A_{l+1} = tanh(Z_{l+1})    (TG_FWD)
//   output layer    Z_L = W_{L-1} A_{L-1} + b_{L-1}                      (TG_OUT)
//   backward        G_l = (W_l' G_{l+1}) (.) (1 - A_l^2)                (TG_BWD)
//   weight gradient dW_l = G_{l+1} A_l'  (split over the batch)          (TG_WG)
// Operands are split into BF16 hi + lo pairs (x = hi + lo to ~2^-17), and
// each product is the three MMAs hi*hi + hi*lo + lo*hi with FP32
// accumulation in tensor memory; in the BF16 mode (TgArgs::split = 0) only
// the hi tiles are loaded and each product is the one MMA hi*hi (operands
// rounded to BF16, FP32 accumulation), and the epilogues write hi only.  Both operands of every GEMM are K-major:
// the forward and backward GEMMs contract over features, so they read the
// activations / gradients node-major ([node][feature]); the weight gradient
// contracts over the batch, so it reads them feature-major ([feature][node]).
// The epilogues write every activation and gradient in both layouts.
// Tiles: M = 128 rows x N = 128 columns, K in blocks of 32 (64 B swizzle),
// six TMA stages, two TMEM accumulators (256 columns); persistent CTAs; one
// warp issues the TMA copies, one the MMAs, eight run the epilogue.  Each
// GEMM of a training step is one tile per CTA and ~2 GFLOP, so much of its
// time is launch and drain: in the BF16 mode the stages hold hi tiles only
// (96 KB), and the next GEMM's CTAs (programmatic dependent launch) fit
// beside the running ones (half the tensor memory each) and run their
// prologue during its drain; with split operands the stages hold hi + lo
// tiles (192 KB, one CTA per SM: three stages of 32 KB measured slower).
#include <algorithm>
#include <vector>

#include "tc_common.cuh"

namespace rtn {
namespace {

constexpr int TG_KB = 32;
constexpr int TG_THREADS = 320;
constexpr int TG_EPI_WARPS = 8;
constexpr uint32_t TG_SBO = 512;  // 8 rows x 64 B
constexpr uint32_t TG_SWZ = 4;    // 64 B swizzle
constexpr uint32_t TG_A_BYTES = 128u * TG_KB * 2u;
// N tile NT: 128 columns (twice the tiles of a 512 x batch GEMM, so that
// more SMs pull operands) with six stages; the weight gradient too (with 256
// columns it ran 9% slower per training step: its batch split twice as
// deep, so the Adam launch summed twice the partial products)
template <int NT>
struct Tg {
  static constexpr uint32_t B_BYTES = (uint32_t)NT * TG_KB * 2u;
  static constexpr uint32_t STAGE = 2u * TG_A_BYTES + 2u * B_BYTES;  // hi + lo tiles
  static constexpr uint32_t STAGE1 = TG_A_BYTES + B_BYTES;             // hi tiles
  static constexpr int STAGES = 6;
  static constexpr size_t SMEM = STAGES * STAGE + 1024 + 512;     // split operands
  static constexpr size_t SMEM1 = STAGES * STAGE1 + 1024 + 512;   // BF16 mode
  static constexpr uint32_t TMEM_COLS = 2 * NT;
};
static_assert(Tg<128>::SMEM <= 232448 && 2 * (Tg<128>::SMEM1 + 1024) <= 233472, "shared memory");

enum { TG_FWD = 0, TG_OUT = 1, TG_BWD = 2, TG_WG = 3 };
// N tile of the weight gradient
constexpr int TG_WG_NT = 128;

struct TgMaps {
  CUtensorMap ah, al, bh, bl;
};

struct TgArgs {
  int m_rows, n_cols;   // real output rows / columns
  int mts, nts, nkb;    // M tiles, N tiles, K blocks per tile
  int ksplit;           // TG_WG: K ranges (one partial product each)
  int split;            // 1: hi + lo operands, three MMAs; 0: hi only, one MMA
  const float* bias;    // TG_FWD, TG_OUT: [m_rows]
  // TG_FWD / TG_BWD outputs: node-major [node][ldn] and feature-major
  // [row][ldf], BF16 hi + lo; columns n >= n_cols of the feature-major rows
  // are written as 0 (the zero padding of the weight gradient's K)
  __nv_bfloat16 *ynh, *ynl, *yfh, *yfl;
  int ldn, ldf;
  // TG_BWD: the layer's activations A_l feature-major [row][ldf], hi + lo
  const __nv_bfloat16 *afh, *afl;
  // TG_BWD: the bias gradient of the produced layer, sum over the batch of
  // G_l, accumulated atomically (zeroed before the step)
  float* db;
  float* out;  // TG_OUT: Z [node][m_rows]; TG_WG: partials [ksplit][m_rows][n_cols]
  int* err;
};

template <int MODE, int NT>
__global__ void __launch_bounds__(TG_THREADS, 1) tg_kernel(const __grid_constant__ TgMaps mp, TgArgs a) {
  constexpr int TG_N = NT, TG_STAGES = Tg<NT>::STAGES;
  constexpr uint32_t TG_B_BYTES = Tg<NT>::B_BYTES;
  // a stage holds hi + lo tiles with split operands, hi tiles otherwise
  const uint32_t TG_STAGE = a.split ? Tg<NT>::STAGE : Tg<NT>::STAGE1;
  const uint32_t b_off = a.split ? 2u * TG_A_BYTES : TG_A_BYTES;  // B hi within a stage
  extern __shared__ uint8_t smem_raw[];
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (sraw & 1023u)) & 1023u;
  uint8_t* sm = smem_raw + pad;
  const uint32_t st0 = sraw + pad;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + TG_STAGES * TG_STAGE);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * TG_STAGES + 5);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  auto bar = [&](int k) { return smem_u32(bars + k); };
  auto full_bar = [&](int s) { return bar(s); };
  auto empty_bar = [&](int s) { return bar(TG_STAGES + s); };
  auto acc_full = [&](int c) { return bar(2 * TG_STAGES + c); };
  auto tmem_free = [&](int c) { return bar(2 * TG_STAGES + 2 + c); };
  const uint32_t mma_done = bar(2 * TG_STAGES + 4);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long n_tiles = (long long)a.mts * a.nts * a.ksplit;

  if (threadIdx.x == 0) {
    for (int s = 0; s < TG_STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int c = 0; c < 2; ++c) {
      mbar_init(acc_full(c), 1);
      mbar_init(tmem_free(c), TG_EPI_WARPS);
    }
    mbar_init(mma_done, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(Tg<NT>::TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  pdl_wait();
  pdl_trigger();

  // tile t: M tile t % mts, N tile (t / mts) % nts, K range t / (mts nts)
  if (warp == 0) {
    // ---------------- TMA producer
    int s = 0;
    uint32_t ph = 0;
    bool ok = true;
    uint32_t issued = 0, last_ph = 0;
    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      const int mt = (int)(t % a.mts), nt = (int)((t / a.mts) % a.nts), ks = (int)(t / ((long long)a.mts * a.nts));
      for (int kb = 0; kb < a.nkb; ++kb) {
        if (!(ok = mbar_wait_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err))) break;
        if (elect_one()) {
          const uint32_t sa = st0 + s * TG_STAGE;
          const int kx = (ks * a.nkb + kb) * TG_KB;
          mbar_expect_tx(full_bar(s), a.split ? TG_STAGE : TG_A_BYTES + TG_B_BYTES);
          tma_load_2d(sa, &mp.ah, kx, mt * 128, full_bar(s));
          tma_load_2d(sa + b_off, &mp.bh, kx, nt * TG_N, full_bar(s));
          if (a.split) {
            tma_load_2d(sa + TG_A_BYTES, &mp.al, kx, mt * 128, full_bar(s));
            tma_load_2d(sa + 2 * TG_A_BYTES + TG_B_BYTES, &mp.bl, kx, nt * TG_N, full_bar(s));
          }
        }
        __syncwarp();
        issued |= 1u << s;
        last_ph = (last_ph & ~(1u << s)) | (ph << s);
        if (++s == TG_STAGES) { s = 0; ph ^= 1u; }
      }
    }
    // copies still in flight complete before the CTA may exit
    for (int q = 0; q < TG_STAGES; ++q)
      if (issued & (1u << q)) {
        const long long t0 = clock64();
        while (!mbar_try(full_bar(q), (last_ph >> q) & 1u) && clock64() - t0 < WAIT_CYCLES) {
        }
      }
  } else if (warp == 1) {
    // ---------------- MMA issuer: hi*hi (+ hi*lo + lo*hi when split) per K step
    constexpr uint32_t idesc = idesc_bf16(128, TG_N);
    int s = 0, acc = 0;
    uint32_t ph = 0, aph = 0;
    bool ok = true;
    for (long long t = blockIdx.x; t < n_tiles && ok; t += gridDim.x) {
      if (!(ok = mbar_wait_warp(tmem_free(acc), aph ^ 1u, abort_flag, a.err))) break;
      tc_fence_after();
      const uint32_t d = tmem + acc * (uint32_t)NT;
      for (int kb = 0; kb < a.nkb; ++kb) {
        if (!(ok = mbar_wait_warp(full_bar(s), ph, abort_flag, a.err))) break;
        tc_fence_after();
        const uint32_t sa = st0 + s * TG_STAGE;
#pragma unroll
        for (int k = 0; k < TG_KB / 16; ++k) {
          const uint64_t ah = kmajor_desc(sa + k * 32u, TG_SBO, TG_SWZ);
          const uint64_t al = kmajor_desc(sa + TG_A_BYTES + k * 32u, TG_SBO, TG_SWZ);
          const uint64_t bh = kmajor_desc(sa + b_off + k * 32u, TG_SBO, TG_SWZ);
          const uint64_t bl = kmajor_desc(sa + 2 * TG_A_BYTES + TG_B_BYTES + k * 32u, TG_SBO, TG_SWZ);
          mma_bf16_elect(d, ah, bh, idesc, (kb | k) != 0);
          if (a.split) {
            mma_bf16_elect(d, ah, bl, idesc, 1u);
            mma_bf16_elect(d, al, bh, idesc, 1u);
          }
        }
        mma_commit_elect(empty_bar(s));
        if (++s == TG_STAGES) { s = 0; ph ^= 1u; }
      }
      if (!ok) break;
      mma_commit_elect(acc_full(acc));
      if (++acc == 2) { acc = 0; aph ^= 1u; }
    }
    mma_commit_elect(mma_done);
    const long long t0 = clock64();
    while (!mbar_try(mma_done, 0) && clock64() - t0 < WAIT_CYCLES) {
    }
  } else {
    // ---------------- epilogue: lane quarter warp % 4 (output row i per
    // lane); the two warps of a quarter take alternate 16-column chunks
    const int q = warp & 3, half = (warp - 2) >> 2;
    int acc = 0;
    uint32_t aph = 0;
    for (long long t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      const int mt = (int)(t % a.mts), nt = (int)((t / a.mts) % a.nts), ks = (int)(t / ((long long)a.mts * a.nts));
      const int i = mt * 128 + q * 32 + lane;
      const bool row_ok = i < a.m_rows;
      float rsum = 0.0f;  // TG_BWD: the lane's row summed over its columns
      const float bi = (MODE == TG_FWD || MODE == TG_OUT) && row_ok ? __ldg(a.bias + i) : 0.0f;
      if (!mbar_wait_warp(acc_full(acc), aph, abort_flag, a.err)) break;
      tc_fence_after();
      const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + acc * (uint32_t)NT;
      for (int ch = half; ch < TG_N / 16; ch += 2) {
        // every lane runs the tensor-memory loads (warp-collective); only
        // the stores depend on the lane's row
        const int j0 = nt * TG_N + 16 * ch;
        float v[16];
        tmem_ld16(taddr + 16 * ch, v);
        // TG_BWD: d = 1 - a^2 of the 16 nodes from the feature-major activations
        uint4 pa[4];
        if (MODE == TG_BWD) {
          const int ir = row_ok ? i : 0;
          const uint4* h4 = reinterpret_cast<const uint4*>(a.afh + (size_t)ir * a.ldf + j0);
          const uint4* l4 = reinterpret_cast<const uint4*>(a.afl + (size_t)ir * a.ldf + j0);
          pa[0] = h4[0]; pa[1] = h4[1];
          if (a.split) {
            pa[2] = l4[0]; pa[3] = l4[1];
          } else {
            pa[2] = pa[3] = make_uint4(0u, 0u, 0u, 0u);
          }
        }
        tmem_wait_ld();
        if (MODE == TG_WG) {
          if (row_ok) {
            float* o = a.out + ((size_t)ks * a.m_rows + i) * a.n_cols + j0;
            if ((a.n_cols & 3) == 0 && j0 + 16 <= a.n_cols) {
#pragma unroll
              for (int k = 0; k < 4; ++k)
                reinterpret_cast<float4*>(o)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
            } else {
#pragma unroll
              for (int k = 0; k < 16; ++k)
                if (j0 + k < a.n_cols) o[k] = v[k];
            }
          }
        } else if (MODE == TG_OUT) {
          if (row_ok) {
#pragma unroll
            for (int k = 0; k < 16; ++k)
              if (j0 + k < a.n_cols) a.out[(size_t)(j0 + k) * a.m_rows + i] = v[k] + bi;
          }
        } else {
          if (MODE == TG_FWD) {
#pragma unroll
            for (int k = 0; k < 16; ++k) v[k] += bi;
            tanh_batch<16>(v);
          } else {
            const __nv_bfloat16* eh = reinterpret_cast<const __nv_bfloat16*>(&pa[0]);
            const __nv_bfloat16* el = reinterpret_cast<const __nv_bfloat16*>(&pa[2]);
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const float av = __bfloat162float(eh[k]) + __bfloat162float(el[k]);
              v[k] *= 1.0f - av * av;
            }
          }
          // columns past the batch become 0 in the feature-major copy
#pragma unroll
          for (int k = 0; k < 16; ++k)
            if (j0 + k >= a.n_cols) v[k] = 0.0f;
          if (MODE == TG_BWD) {
#pragma unroll
            for (int k = 0; k < 16; ++k) rsum += v[k];
          }
          uint32_t hp[8], lp[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            hp[k] = pack_bf16(v[2 * k], v[2 * k + 1]);
            lp[k] = pack_res(v[2 * k], v[2 * k + 1], hp[k]);
          }
          if (row_ok) {
            uint4* fh = reinterpret_cast<uint4*>(a.yfh + (size_t)i * a.ldf + j0);
            uint4* fl = reinterpret_cast<uint4*>(a.yfl + (size_t)i * a.ldf + j0);
            fh[0] = make_uint4(hp[0], hp[1], hp[2], hp[3]);
            fh[1] = make_uint4(hp[4], hp[5], hp[6], hp[7]);
            if (a.split) {
              fl[0] = make_uint4(lp[0], lp[1], lp[2], lp[3]);
              fl[1] = make_uint4(lp[4], lp[5], lp[6], lp[7]);
            }
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              if (j0 + k < a.n_cols) {
                const uint32_t hw = hp[k >> 1] >> (16 * (k & 1)), lw = lp[k >> 1] >> (16 * (k & 1));
                const size_t o = (size_t)(j0 + k) * a.ldn + i;
                reinterpret_cast<uint16_t*>(a.ynh)[o] = (uint16_t)(hw & 0xffffu);
                if (a.split) reinterpret_cast<uint16_t*>(a.ynl)[o] = (uint16_t)(lw & 0xffffu);
              }
            }
          }
        }
        __syncwarp();
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_free(acc));
      if (++acc == 2) { acc = 0; aph ^= 1u; }
      if (MODE == TG_BWD && a.db && row_ok) atomicAdd(a.db + i, rsum);
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Tg<NT>::TMEM_COLS)
                 : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult qr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &qr) ==
            cudaSuccess &&
        p && qr == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// One planned GEMM of the training step (operand tensor maps and epilogue).
struct TgGemm {
  int mode = 0;
  int nt = 256;  // N tile
  TgMaps maps;
  TgArgs args;
  int grid = 0;
};

// K-major BF16 operand [rows][ld] (rows a multiple of the box height, ld and
// k_extent multiples of 32): tensor map with a 32 x box_rows box, 64 B swizzle
bool tg_map(CUtensorMap* m, const __nv_bfloat16* p, long long rows, int k_extent, int ld, int box_rows) {
  auto enc = encoder();
  if (!enc) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)k_extent, (cuuint64_t)rows};
  const cuuint64_t str[1] = {(cuuint64_t)ld * 2};
  const cuuint32_t box[2] = {(cuuint32_t)TG_KB, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<__nv_bfloat16*>(p), dims, str, box, estr,
             CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Plan one GEMM C[m_rows][n_cols] = A B' with A [rows_a][k] (hi, lo) and B
// [rows_b][k] (hi, lo), both K-major; k_blocks K blocks of 32 in total,
// split into ksplit ranges (TG_WG only).  Returns false if a tensor map
// cannot be encoded.
bool tg_plan(TgGemm& g, int mode, const __nv_bfloat16* ah, const __nv_bfloat16* al, long long rows_a,
             int lda, const __nv_bfloat16* bh, const __nv_bfloat16* bl, long long rows_b, int ldb, int k_blocks,
             int m_rows, int n_cols, int n_sm, bool split) {
  g.mode = mode;
  g.nt = mode == TG_WG ? TG_WG_NT : 128;
  TgArgs& a = g.args;
  a = TgArgs{};
  a.split = split ? 1 : 0;
  a.m_rows = m_rows;
  a.n_cols = n_cols;
  a.mts = (m_rows + 127) / 128;
  a.nts = (n_cols + g.nt - 1) / g.nt;
  a.ksplit = 1;
  a.nkb = k_blocks;
  if (mode == TG_WG) {
    // split the batch so that about one tile per SM runs
    const int base = a.mts * a.nts;
    const int want = std::max(1, std::min(k_blocks, n_sm / std::max(base, 1)));
    a.nkb = (k_blocks + want - 1) / want;
    a.ksplit = (k_blocks + a.nkb - 1) / a.nkb;
  }
  const int kx = k_blocks * TG_KB;
  if (!tg_map(&g.maps.ah, ah, rows_a, kx, lda, 128) || !tg_map(&g.maps.al, al, rows_a, kx, lda, 128) ||
      !tg_map(&g.maps.bh, bh, rows_b, kx, ldb, g.nt) || !tg_map(&g.maps.bl, bl, rows_b, kx, ldb, g.nt))
    return false;
  g.grid = (int)std::min<long long>((long long)a.mts * a.nts * a.ksplit, std::max(1, n_sm));
  return true;
}

// dynamic shared memory of the four GEMM kernels, and the whole carveout as
// shared memory so that two CTAs (the running GEMM's and the next one's)
// fit on an SM
template <typename K>
cudaError_t tg_attrs(K* k, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k, cudaFuncAttributePreferredSharedMemoryCarveout, cudaSharedmemCarveoutMaxShared);
  return e;
}

cudaError_t tg_setup() {
  cudaError_t e;
  if ((e = tg_attrs(tg_kernel<TG_FWD, 128>, Tg<128>::SMEM))) return e;
  if ((e = tg_attrs(tg_kernel<TG_OUT, 128>, Tg<128>::SMEM))) return e;
  if ((e = tg_attrs(tg_kernel<TG_BWD, 128>, Tg<128>::SMEM))) return e;
  return tg_attrs(tg_kernel<TG_WG, TG_WG_NT>, Tg<TG_WG_NT>::SMEM);
}

// err: the context's device status word (re-read at every launch: the
// network packs, and with them the word, are rebuilt after training)
cudaError_t tg_launch(const TgGemm& g, int* err, cudaStream_t s) {
  TgArgs a = g.args;
  a.err = err;
  const size_t sm = a.split ? Tg<128>::SMEM : Tg<128>::SMEM1;
  static_assert(TG_WG_NT == 128, "one shared-memory size for the four kernels");
  switch (g.mode) {
    case TG_FWD: return launch_pdl(tg_kernel<TG_FWD, 128>, dim3(g.grid), dim3(TG_THREADS), sm, s, g.maps, a);
    case TG_OUT: return launch_pdl(tg_kernel<TG_OUT, 128>, dim3(g.grid), dim3(TG_THREADS), sm, s, g.maps, a);
    case TG_BWD: return launch_pdl(tg_kernel<TG_BWD, 128>, dim3(g.grid), dim3(TG_THREADS), sm, s, g.maps, a);
    default: return launch_pdl(tg_kernel<TG_WG, TG_WG_NT>, dim3(g.grid), dim3(TG_THREADS), sm, s, g.maps, a);
  }
}

// epilogue operands of a planned GEMM
void tg_set_out(TgGemm& g, const float* bias, __nv_bfloat16* ynh, __nv_bfloat16* ynl, int ldn, __nv_bfloat16* yfh,
                __nv_bfloat16* yfl, int ldf, const __nv_bfloat16* afh, const __nv_bfloat16* afl, float* out, int* err,
                float* db = nullptr) {
  TgArgs& a = g.args;
  a.db = db;
  a.bias = bias;
  a.ynh = ynh; a.ynl = ynl; a.ldn = ldn;
  a.yfh = yfh; a.yfl = yfl; a.ldf = ldf;
  a.afh = afh; a.afl = afl;
  a.out = out;
  a.err = err;
}

int tg_ksplit(const TgGemm& g) { return g.args.ksplit; }

inline int rup(int x, int m) { return (x + m - 1) / m * m; }
inline unsigned nblk(size_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }


__device__ __forceinline__ void split2(float v, __nv_bfloat16& h, __nv_bfloat16& l) {
  h = __float2bfloat16_rn(v);
  l = __float2bfloat16_rn(v - __bfloat162float(h));
}

// z = [x; u] of samples start .. start + bs - 1 as A_0: node-major [rows][32]
// (features 17..31 zero) and feature-major [17][ldf]; samples j >= bs are 0.
// In a replayed training step it also advances the Adam step counter t_inc,
// which only the step's Adam launch, several launches later, reads.
__global__ void tg_gather_kernel(const float* __restrict__ X, const float* __restrict__ U, int start, int bs,
                                 int ldf, __nv_bfloat16* __restrict__ nh, __nv_bfloat16* __restrict__ nl,
                                 __nv_bfloat16* __restrict__ fh, __nv_bfloat16* __restrict__ fl,
                                 const int* __restrict__ k_dev, int per_epoch, float* __restrict__ db, int nb,
                                 int* __restrict__ t_inc) {
  pdl_wait();
  pdl_trigger();
  if (t_inc && blockIdx.x == 0 && threadIdx.x == 0) *t_inc += 1;
  // the bias gradients, which the loss and backward launches accumulate
  for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < nb; e += (long long)gridDim.x * blockDim.x)
    db[e] = 0.0f;
  // a replayed step: its minibatch from the step counter on the device
  if (k_dev) start = (*k_dev % per_epoch) * bs;
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (long long)ldf * 32) return;
  const int j = (int)(e >> 5), f = (int)(e & 31);
  float v = 0.0f;
  if (j < bs && f < NZ) {
    const size_t r = (size_t)start + j;
    v = f < NX ? X[r * NX + f] : U[r * NU + (f - NX)];
  }
  __nv_bfloat16 h, l;
  split2(v, h, l);
  nh[(size_t)j * 32 + f] = h;
  nl[(size_t)j * 32 + f] = l;
  if (f < NZ) {
    fh[(size_t)f * ldf + j] = h;
    fl[(size_t)f * ldf + j] = l;
  }
}

// G_L = 2 (Z - Y) / (no bs) (loss 1/(no bs) sum (Z - Y)^2): node-major
// [rows][32] (columns >= no zero) and feature-major [no][ldf] (samples
// j >= bs zero); the loss summed per block into *loss, and the output
// layer's bias gradient (G_L summed over the batch) per block into db
__global__ void tg_loss_kernel(const float* __restrict__ Z, const float* __restrict__ Y, int start, int bs, int no,
                               int ldf, __nv_bfloat16* __restrict__ nh, __nv_bfloat16* __restrict__ nl,
                               __nv_bfloat16* __restrict__ fh, __nv_bfloat16* __restrict__ fl, float* loss,
                               float* __restrict__ db, const int* __restrict__ k_dev, int per_epoch) {
  pdl_wait();
  pdl_trigger();
  // a replayed step: its minibatch and loss entry from the step counter on the device
  if (k_dev) {
    start = (*k_dev % per_epoch) * bs;
    loss += *k_dev;
  }
  __shared__ float red[256];
  __shared__ float rsum[32];
  if (threadIdx.x < 32) rsum[threadIdx.x] = 0.0f;
  __syncthreads();
  const long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  float e2 = 0.0f;
  if (e < (long long)ldf * 32) {
    const int j = (int)(e >> 5), r = (int)(e & 31);
    float g = 0.0f;
    if (j < bs && r < no) {
      const float d = Z[(size_t)j * no + r] - Y[((size_t)start + j) * no + r];
      g = 2.0f * d / ((float)no * bs);
      e2 = d * d;
    }
    __nv_bfloat16 h, l;
    split2(g, h, l);
    nh[(size_t)j * 32 + r] = h;
    nl[(size_t)j * 32 + r] = l;
    if (r < no) {
      fh[(size_t)r * ldf + j] = h;
      fl[(size_t)r * ldf + j] = l;
      atomicAdd(&rsum[r], g);
    }
  }
  red[threadIdx.x] = e2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] / ((float)no * bs));
  if (threadIdx.x < no) atomicAdd(db + threadIdx.x, rsum[threadIdx.x]);
}

// weight-gradient partials of one layer summed: g[e] = sum_s part[s][e]
__global__ void tg_reduce_kernel(const float* __restrict__ part, int ks, size_t n, float* __restrict__ g) {
  const size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n) return;
  float s = 0.0f;
  for (int k = 0; k < ks; ++k) s += part[(size_t)k * n + e];
  g[e] = s;
}

__device__ __forceinline__ float adam_elem(float p, float g, float& m, float& v, float lr, float b1, float b2,
                                           float eps, float c1, float c2) {
  m = b1 * m + (1.0f - b1) * g;
  v = b2 * v + (1.0f - b2) * g * g;
  return p - lr * (m / c1) / (sqrtf(v / c2) + eps);
}

// one layer's Adam + repack job (the per-step launch covers every layer)
struct WJob {
  float* P;            // W_l [fo][fi] (FP32 master)
  const float* part;   // weight-gradient partials [ks][fo][fi]
  float *m, *v;        // Adam moments of W_l
  __nv_bfloat16 *wh, *wl, *th, *tl;
  int ks, fo, fi, ldw, ldwt;
  int bx, blk0;        // 32-column tiles per row of tiles; first block of the layer
};

// one 32 x 32 tile of a layer's weights W [fo][fi], 256 threads, four
// consecutive elements of a row per thread (float4 loads where the row length
// allows): with adam, the Adam step from the summed partials; then the split
// copies W (hi, lo) [fo][ldw] and W' (hi, lo) [fi][ldwt], the transpose
// through shared memory so that both copies are stored as 8-byte runs
__device__ __forceinline__ void weights_tile(const WJob& J, int bx, int by, int adam, float lr, float b1, float b2,
                                             float eps, float c1, float c2) {
  __shared__ uint32_t tile[32][33];  // hi | lo << 16
  float* __restrict__ P = J.P;
  const float* __restrict__ part = J.part;
  float* __restrict__ m = J.m;
  float* __restrict__ v = J.v;
  const int fo = J.fo, fi = J.fi, ks = J.ks, ldw = J.ldw, ldwt = J.ldwt;
  const size_t n = (size_t)fo * fi;
  const int r = threadIdx.x >> 3, c4 = (threadIdx.x & 7) * 4;
  const int i = by * 32 + r, j = bx * 32 + c4;
  float pv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
  if (i < fo && j < fi) {
    const size_t e = (size_t)i * fi + j;
    if ((fi & 3) == 0) {  // j + 3 < fi and 16-byte aligned
      float4 p4 = *reinterpret_cast<const float4*>(P + e);
      pv[0] = p4.x; pv[1] = p4.y; pv[2] = p4.z; pv[3] = p4.w;
      if (adam) {
        float4 g4 = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
#pragma unroll 6
        for (int q = 0; q < ks; ++q) {
          const float4 x = *reinterpret_cast<const float4*>(part + (size_t)q * n + e);
          g4.x += x.x; g4.y += x.y; g4.z += x.z; g4.w += x.w;
        }
        float4 m4 = *reinterpret_cast<const float4*>(m + e), v4 = *reinterpret_cast<const float4*>(v + e);
        pv[0] = adam_elem(pv[0], g4.x, m4.x, v4.x, lr, b1, b2, eps, c1, c2);
        pv[1] = adam_elem(pv[1], g4.y, m4.y, v4.y, lr, b1, b2, eps, c1, c2);
        pv[2] = adam_elem(pv[2], g4.z, m4.z, v4.z, lr, b1, b2, eps, c1, c2);
        pv[3] = adam_elem(pv[3], g4.w, m4.w, v4.w, lr, b1, b2, eps, c1, c2);
        *reinterpret_cast<float4*>(m + e) = m4;
        *reinterpret_cast<float4*>(v + e) = v4;
        *reinterpret_cast<float4*>(P + e) = make_float4(pv[0], pv[1], pv[2], pv[3]);
      }
    } else {
      for (int k = 0; k < 4 && j + k < fi; ++k) {
        float p = P[e + k];
        if (adam) {
          float g = 0.0f;
          for (int q = 0; q < ks; ++q) g += part[(size_t)q * n + e + k];
          p = adam_elem(p, g, m[e + k], v[e + k], lr, b1, b2, eps, c1, c2);
          P[e + k] = p;
        }
        pv[k] = p;
      }
    }
  }
  uint32_t hw[2] = {0u, 0u}, lw[2] = {0u, 0u};
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    __nv_bfloat16 h, l;
    split2(pv[k], h, l);
    const uint32_t hb = __bfloat16_as_ushort(h), lb = __bfloat16_as_ushort(l);
    hw[k >> 1] |= hb << (16 * (k & 1));
    lw[k >> 1] |= lb << (16 * (k & 1));
    tile[r][c4 + k] = hb | (lb << 16);
  }
  if (i < fo && j < fi) {
    if ((fi & 3) == 0) {  // ldw is a multiple of 32: 8-byte aligned runs
      *reinterpret_cast<uint2*>(J.wh + (size_t)i * ldw + j) = make_uint2(hw[0], hw[1]);
      *reinterpret_cast<uint2*>(J.wl + (size_t)i * ldw + j) = make_uint2(lw[0], lw[1]);
    } else {
      for (int k = 0; k < 4 && j + k < fi; ++k) {
        J.wh[(size_t)i * ldw + j + k] = __ushort_as_bfloat16((unsigned short)(tile[r][c4 + k] & 0xffffu));
        J.wl[(size_t)i * ldw + j + k] = __ushort_as_bfloat16((unsigned short)(tile[r][c4 + k] >> 16));
      }
    }
  }
  __syncthreads();
  // W': row jt = column j of W, four consecutive rows of W per thread
  const int jt = bx * 32 + r, it = by * 32 + c4;
  if (jt < fi && it < fo) {
    uint32_t th2[2] = {0u, 0u}, tl2[2] = {0u, 0u};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t pk = tile[c4 + k][r];
      th2[k >> 1] |= (pk & 0xffffu) << (16 * (k & 1));
      tl2[k >> 1] |= (pk >> 16) << (16 * (k & 1));
    }
    if (it + 3 < fo) {  // ldwt is a multiple of 32
      *reinterpret_cast<uint2*>(J.th + (size_t)jt * ldwt + it) = make_uint2(th2[0], th2[1]);
      *reinterpret_cast<uint2*>(J.tl + (size_t)jt * ldwt + it) = make_uint2(tl2[0], tl2[1]);
    } else {
      for (int k = 0; it + k < fo; ++k) {
        const uint32_t pk = tile[c4 + k][r];
        J.th[(size_t)jt * ldwt + it + k] = __ushort_as_bfloat16((unsigned short)(pk & 0xffffu));
        J.tl[(size_t)jt * ldwt + it + k] = __ushort_as_bfloat16((unsigned short)(pk >> 16));
      }
    }
  }
}

// the BF16 copies of one layer's weights from its FP32 master (no Adam)
__global__ void __launch_bounds__(256) tg_split_kernel(WJob J) {
  weights_tile(J, blockIdx.x, blockIdx.y, 0, 0.f, 0.f, 0.f, 0.f, 1.f, 1.f);
}

// Adam of the biases: element i of n
__device__ __forceinline__ void bias_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ m,
                                          float* __restrict__ v, size_t i, float lr, float b1, float b2, float eps,
                                          float c1, float c2) {
  const float g = G[i];
  const float mi = b1 * m[i] + (1.0f - b1) * g;
  const float vi = b2 * v[i] + (1.0f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  P[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// The Adam step (bias-corrected, step t) of every layer's weights and of the
// biases in one launch: blocks below wblocks -> (layer, 32 x 32 tile) by the
// jobs' first blocks, the rest -> 256 biases each.  In a replayed step the
// first bias block advances the minibatch counter k_inc for the next replay
// (its readers, the gather and loss launches, ran before this one).
__global__ void __launch_bounds__(256) tg_weights_kernel(const WJob* __restrict__ jobs, int n_jobs, int wblocks,
                                                         float lr, float b1, float b2, float eps,
                                                         const int* __restrict__ t_dev, float* __restrict__ bP,
                                                         const float* __restrict__ bG, float* __restrict__ bm,
                                                         float* __restrict__ bv, int nb, int* __restrict__ k_inc) {
  pdl_wait();
  pdl_trigger();
  const float c1 = 1.0f - powf(b1, (float)*t_dev), c2 = 1.0f - powf(b2, (float)*t_dev);
  if ((int)blockIdx.x >= wblocks) {
    const int bb = (int)blockIdx.x - wblocks;
    if (bb == 0 && threadIdx.x == 0 && k_inc) *k_inc += 1;
    const size_t i = (size_t)bb * blockDim.x + threadIdx.x;
    if (i < (size_t)nb) bias_adam(bP, bG, bm, bv, i, lr, b1, b2, eps, c1, c2);
    return;
  }
  int li = 0;
  while (li + 1 < n_jobs && (int)blockIdx.x >= jobs[li + 1].blk0) ++li;
  const WJob J = jobs[li];
  const int b = (int)blockIdx.x - J.blk0;
  weights_tile(J, b % J.bx, b / J.bx, 1, lr, b1, b2, eps, c1, c2);
}

inline dim3 wgrid(int fo, int fi) { return dim3((unsigned)((fi + 31) / 32), (unsigned)((fo + 31) / 32)); }
const dim3 WBLOCK(256);

// layer l's Adam + repack job (part, ks, m, v are read only with Adam)
WJob weight_job(const Net& net, const TrainState& ts, int l) {
  const std::vector<int>& w = net.widths;
  WJob J;
  J.P = net.W32 + net.w_off[l];
  J.part = ts.part ? ts.part + ts.part_off[l] : nullptr;
  J.ks = ts.ksplit.empty() ? 0 : ts.ksplit[l];
  J.m = ts.m + net.w_off[l];
  J.v = ts.v + net.w_off[l];
  J.wh = ts.ws[4 * l];
  J.wl = ts.ws[4 * l + 1];
  J.th = ts.ws[4 * l + 2];
  J.tl = ts.ws[4 * l + 3];
  J.fo = w[l + 1];
  J.fi = w[l];
  J.ldw = rup(w[l], 32);
  J.ldwt = rup(w[l + 1], 32);
  J.bx = (w[l] + 31) / 32;
  J.blk0 = 0;
  return J;
}

struct TgPlan {
  std::vector<TgGemm> fwd;  // L - 1 hidden layers, then the output layer
  std::vector<TgGemm> wg;   // per layer l
  std::vector<TgGemm> bwd;  // per layer l >= 1 (index l)
};

// batch ranges of the weight gradient of a fo x fi layer for up to cap
// samples (tg_plan never splits a smaller batch into more)
int wg_ksplit_max(int fo, int fi, int cap, int n_sm) {
  const int base = ((fo + 127) / 128) * ((fi + TG_WG_NT - 1) / TG_WG_NT), kb = rup(cap, 32) / 32;
  return std::max(1, std::min(kb, n_sm / std::max(base, 1)));
}

template <typename T>
cudaError_t zalloc(T** p, size_t n) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(n, 1) * sizeof(T));
  if (e == cudaSuccess) e = cudaMemset(*p, 0, std::max<size_t>(n, 1) * sizeof(T));
  return e;
}

void free_bufs(TrainState& ts) {
  for (auto* v : {&ts.an, &ts.af, &ts.gn, &ts.gf})
    for (auto* p : *v) if (p) cudaFree(p);
  ts.an.clear(); ts.af.clear(); ts.gn.clear(); ts.gf.clear();
  if (ts.z) cudaFree(ts.z);
  if (ts.part) cudaFree(ts.part);
  ts.z = nullptr;
  ts.part = nullptr;
  ts.cap = 0;
}

}  // namespace

cudaError_t train_prepare(rtn_ctx* ctx, TrainState& ts, int cap, int bs, std::string& err) {
  Net& net = ctx->net;
  const int L = net.n_layers, no = net.widths[L];
  const int n_sm = std::max(1, ctx->net.tc.n_sm);
  const std::vector<int>& w = net.widths;
  cudaError_t e;
  if (!ts.side) {
    if ((e = cudaStreamCreateWithFlags(&ts.side, cudaStreamNonBlocking))) return e;
    ts.evs.assign(L + 1, nullptr);
    for (auto& ev : ts.evs)
      if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming))) return e;
  }
  if (!ts.grad) {
    ts.nw = ts.nb = 0;
    for (int l = 0; l < L; ++l) {
      ts.nw += (size_t)w[l + 1] * w[l];
      ts.nb += w[l + 1];
    }
    ts.b_base = ts.nw;
    if ((e = zalloc(&ts.grad, ts.nw + ts.nb))) return e;
    if ((e = zalloc(&ts.m, ts.nw + ts.nb))) return e;
    if ((e = zalloc(&ts.v, ts.nw + ts.nb))) return e;
    if ((e = zalloc(&ts.t_dev, 1))) return e;
    ts.t = 0;
    if ((e = tg_setup())) return e;
    // split copies of the weights
    ts.ws.assign(4 * L, nullptr);
    for (int l = 0; l < L; ++l) {
      const size_t nwl = (size_t)rup(w[l + 1], 128) * rup(w[l], 32), ntl = (size_t)rup(w[l], 128) * rup(w[l + 1], 32);
      for (int k = 0; k < 4; ++k)
        if ((e = zalloc(&ts.ws[4 * l + k], k < 2 ? nwl : ntl))) return e;
      tg_split_kernel<<<wgrid(w[l + 1], w[l]), WBLOCK, 0, ctx->stream>>>(weight_job(net, ts, l));
    }
    if ((e = cudaGetLastError())) return e;
  }
  if (ts.cap < cap) {
    free_bufs(ts);
    ts.rows = rup(cap, 256);
    ts.ldf = rup(cap, 256);
    ts.an.assign(2 * L, nullptr); ts.af.assign(2 * L, nullptr);
    ts.gn.assign(2 * L, nullptr); ts.gf.assign(2 * L, nullptr);
    for (int l = 0; l < L; ++l)
      for (int k = 0; k < 2; ++k) {
        if ((e = zalloc(&ts.an[2 * l + k], (size_t)ts.rows * rup(w[l], 32)))) return e;
        if ((e = zalloc(&ts.af[2 * l + k], (size_t)rup(w[l], 256) * ts.ldf))) return e;
        if ((e = zalloc(&ts.gn[2 * l + k], (size_t)ts.rows * rup(w[l + 1], 32)))) return e;
        if ((e = zalloc(&ts.gf[2 * l + k], (size_t)rup(w[l + 1], 256) * ts.ldf))) return e;
      }
    if ((e = zalloc(&ts.z, (size_t)cap * no))) return e;
    // partial products of the weight gradients for the largest batch
    ts.part_off.assign(L + 1, 0);
    ts.ksplit.assign(L, 1);
    size_t tot = 0;
    for (int l = 0; l < L; ++l) {
      ts.part_off[l] = tot;  // 256 B aligned: the epilogue stores float4
      tot += ((size_t)wg_ksplit_max(w[l + 1], w[l], cap, n_sm) * w[l + 1] * w[l] + 63) / 64 * 64;
    }
    ts.part_off[L] = tot;
    if ((e = zalloc(&ts.part, tot))) return e;
    ts.cap = cap;
    ts.bs = 0;
  }
  if (ts.bs == bs && ts.plan) return cudaSuccess;
  // plan of a step on bs samples
  TgPlan* P = static_cast<TgPlan*>(ts.plan);
  if (!P) ts.plan = P = new TgPlan();
  P->fwd.assign(L, TgGemm{});
  P->wg.assign(L, TgGemm{});
  P->bwd.assign(L, TgGemm{});
  int* derr = net.tc.err;
  const bool split = !ctx->opt.train_bf16;
  for (int l = 0; l < L; ++l) {
    const bool out = l == L - 1;
    TgGemm& g = P->fwd[l];
    if (!tg_plan(g, out ? TG_OUT : TG_FWD, ts.ws[4 * l], ts.ws[4 * l + 1], rup(w[l + 1], 128), rup(w[l], 32),
                 ts.an[2 * l], ts.an[2 * l + 1], ts.rows, rup(w[l], 32), rup(w[l], 32) / 32, w[l + 1], bs, n_sm, split)) {
      err = "training: tensor map encoding failed";
      return cudaSuccess;
    }
    if (out)
      tg_set_out(g, net.b32 + net.b_off[l], nullptr, nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, ts.z, derr);
    else
      tg_set_out(g, net.b32 + net.b_off[l], ts.an[2 * (l + 1)], ts.an[2 * (l + 1) + 1], rup(w[l + 1], 32),
                 ts.af[2 * (l + 1)], ts.af[2 * (l + 1) + 1], ts.ldf, nullptr, nullptr, nullptr, derr);
    // dW_l = G_{l+1} A_l' over the batch
    TgGemm& gw = P->wg[l];
    if (!tg_plan(gw, TG_WG, ts.gf[2 * l], ts.gf[2 * l + 1], rup(w[l + 1], 256), ts.ldf, ts.af[2 * l],
                 ts.af[2 * l + 1], rup(w[l], 256), ts.ldf, rup(bs, 32) / 32, w[l + 1], w[l], n_sm, split)) {
      err = "training: tensor map encoding failed";
      return cudaSuccess;
    }
    tg_set_out(gw, nullptr, nullptr, nullptr, 0, nullptr, nullptr, 0, nullptr, nullptr, ts.part + ts.part_off[l], derr);
    if ((size_t)tg_ksplit(gw) * w[l + 1] * w[l] > ts.part_off[l + 1] - ts.part_off[l]) {
      err = "training: weight-gradient partials exceed their buffer";
      return cudaSuccess;
    }
    ts.ksplit[l] = tg_ksplit(gw);
    // G_l = (W_l' G_{l+1}) (.) (1 - A_l^2)
    if (l >= 1) {
      TgGemm& gb = P->bwd[l];
      if (!tg_plan(gb, TG_BWD, ts.ws[4 * l + 2], ts.ws[4 * l + 3], rup(w[l], 128), rup(w[l + 1], 32), ts.gn[2 * l],
                   ts.gn[2 * l + 1], ts.rows, rup(w[l + 1], 32), rup(w[l + 1], 32) / 32, w[l], bs, n_sm, split)) {
        err = "training: tensor map encoding failed";
        return cudaSuccess;
      }
      tg_set_out(gb, nullptr, ts.gn[2 * (l - 1)], ts.gn[2 * (l - 1) + 1], rup(w[l], 32), ts.gf[2 * (l - 1)],
                 ts.gf[2 * (l - 1) + 1], ts.ldf, ts.af[2 * l], ts.af[2 * l + 1], nullptr, derr,
                 ts.grad + ts.b_base + net.b_off[l - 1]);
    }
  }
  // the Adam jobs of every layer, for the one per-step launch
  {
    std::vector<WJob> jobs(L);
    int blk = 0;
    for (int l = 0; l < L; ++l) {
      jobs[l] = weight_job(net, ts, l);
      jobs[l].blk0 = blk;
      blk += jobs[l].bx * ((w[l + 1] + 31) / 32);
    }
    if (!ts.wjobs && (e = cudaMalloc(&ts.wjobs, sizeof(WJob) * L))) return e;
    if ((e = cudaMemcpy(ts.wjobs, jobs.data(), sizeof(WJob) * L, cudaMemcpyHostToDevice))) return e;
    ts.wjob_blocks = blk;
  }
  ts.bs = bs;
  return cudaSuccess;
}

static cudaError_t grad_impl(rtn_ctx* ctx, TrainState& ts, const float* X, const float* U, const float* Y,
                             int start, float* loss, const int* k_dev, int per_epoch);

cudaError_t train_grad(rtn_ctx* ctx, TrainState& ts, const float* X, const float* U, const float* Y, int start,
                       float* loss) {
  return grad_impl(ctx, ts, X, U, Y, start, loss, nullptr, 1);
}

cudaError_t train_grad_dev(rtn_ctx* ctx, TrainState& ts, const float* X, const float* U, const float* Y,
                           const int* k_dev, int per_epoch, float* losses) {
  return grad_impl(ctx, ts, X, U, Y, 0, losses, k_dev, per_epoch);
}

static cudaError_t grad_impl(rtn_ctx* ctx, TrainState& ts, const float* X, const float* U, const float* Y,
                             int start, float* loss, const int* k_dev, int per_epoch) {
  Net& net = ctx->net;
  const int L = net.n_layers, no = net.widths[L], bs = ts.bs;
  const TgPlan* P = static_cast<const TgPlan*>(ts.plan);
  if (!P) return cudaErrorInvalidValue;
  cudaStream_t s = ctx->stream;
  cudaError_t e;
  // the gather also zeroes the bias gradients, which the loss and backward
  // launches accumulate atomically
  if ((e = launch_pdl(tg_gather_kernel, dim3(nblk((size_t)ts.ldf * 32)), dim3(256), 0, s, X, U, start, bs, ts.ldf,
                      ts.an[0], ts.an[1], ts.af[0], ts.af[1], k_dev, per_epoch, ts.grad + ts.b_base, (int)ts.nb,
                      k_dev ? ts.t_dev : nullptr)))
    return e;
  for (int l = 0; l < L; ++l)
    if ((e = tg_launch(P->fwd[l], net.tc.err, s))) return e;
  if ((e = launch_pdl(tg_loss_kernel, dim3(nblk((size_t)ts.ldf * 32)), dim3(256), 0, s, (const float*)ts.z, Y, start,
                      bs, no, ts.ldf, ts.gn[2 * (L - 1)], ts.gn[2 * (L - 1) + 1], ts.gf[2 * (L - 1)],
                      ts.gf[2 * (L - 1) + 1], loss, ts.grad + ts.b_base + net.b_off[L - 1], k_dev, per_epoch)))
    return e;
  // the weight gradient of layer l (dW_l = G_{l+1} A_l') and the backward
  // GEMM below it (G_l) read only G_{l+1}: the weight gradients go to the
  // side stream, forked once G_{l+1} is complete, joined before the return
  for (int l = L - 1; l >= 0; --l) {
    if ((e = cudaEventRecord(ts.evs[l], s))) return e;
    if ((e = cudaStreamWaitEvent(ts.side, ts.evs[l], 0))) return e;
    if ((e = tg_launch(P->wg[l], net.tc.err, ts.side))) return e;
    if (l >= 1 && (e = tg_launch(P->bwd[l], net.tc.err, s))) return e;
  }
  if ((e = cudaEventRecord(ts.evs[L], ts.side))) return e;
  if ((e = cudaStreamWaitEvent(s, ts.evs[L], 0))) return e;
  return cudaGetLastError();
}

cudaError_t train_reduce(rtn_ctx* ctx, TrainState& ts) {
  Net& net = ctx->net;
  for (int l = 0; l < net.n_layers; ++l) {
    const size_t n = (size_t)net.widths[l + 1] * net.widths[l];
    tg_reduce_kernel<<<nblk(n), 256, 0, ctx->stream>>>(ts.part + ts.part_off[l], ts.ksplit[l], n,
                                                       ts.grad + net.w_off[l]);
  }
  return cudaGetLastError();
}

// The Adam step of a replayed training step: the step counter on the device
// (so that a captured step can be replayed) was advanced by the step's
// gather launch; one launch updates every weight matrix and the biases and
// advances the minibatch counter k_dev for the next replay.
cudaError_t train_adam(rtn_ctx* ctx, TrainState& ts, float lr, int* k_dev) {
  Net& net = ctx->net;
  ts.t += 1;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  return launch_pdl(tg_weights_kernel, dim3(ts.wjob_blocks + nblk(ts.nb)), WBLOCK, 0, ctx->stream,
                    static_cast<const WJob*>(ts.wjobs), net.n_layers, ts.wjob_blocks, lr, b1, b2, eps,
                    (const int*)ts.t_dev, net.b32, (const float*)(ts.grad + ts.b_base), ts.m + ts.nw,
                    ts.v + ts.nw, (int)ts.nb, k_dev);
}

cudaError_t train_resplit(rtn_ctx* ctx, TrainState& ts) {
  Net& net = ctx->net;
  const std::vector<int>& w = net.widths;
  if (ts.ws.empty()) return cudaSuccess;
  for (int l = 0; l < net.n_layers; ++l)
    tg_split_kernel<<<wgrid(w[l + 1], w[l]), WBLOCK, 0, ctx->stream>>>(weight_job(net, ts, l));
  return cudaGetLastError();
}

void train_release(rtn_ctx* ctx) {
  TrainState& ts = ctx->train;
  for (cudaEvent_t ev : ts.evs)
    if (ev) cudaEventDestroy(ev);
  if (ts.side) cudaStreamDestroy(ts.side);
  free_bufs(ts);
  for (auto* p : ts.ws) if (p) cudaFree(p);
  for (void* p : {(void*)ts.grad, (void*)ts.m, (void*)ts.v, (void*)ts.t_dev, ts.wjobs}) if (p) cudaFree(p);
  delete static_cast<TgPlan*>(ts.plan);
  ts = TrainState{};
}

}  // namespace rtn
