// mlp_tc.cu -- (a1) residual network value + forward-mode input Jacobian on the
// 5th-generation tensor cores (tcgen05), one fused kernel for all layers.
//
// Forward mode (Sec. III-A, Eq. 4): every node carries 18 columns through the
// network (its value and the 17 tangent directions d/d[x; u]).  A CTA owns
// NPC nodes; their columns stay on chip for the whole network:
//   * the layer input X (K = hidden width, N = node columns) lives in shared
//     memory as the N-major, unswizzled B operand of tcgen05.mma, in BF16
//     (RTN_BF16) or as a BF16 hi + lo pair (RTN_BF16X2: X = hi + lo, ~16
//     significant bits), either in two buffers with two MMAs per K step
//     (mode 1) or side by side along N in one MMA of twice the width whose
//     two accumulator halves the epilogue adds (mode 2);
//   * the weights W_l (M = output neurons, K-major) stream from L2 by TMA in
//     128 x 64 tiles (128B swizzle) through an mbarrier pipeline;
//   * the accumulators of all output neurons (M tiles of 128 lanes x N
//     columns, FP32) sit in tensor memory;
//   * the epilogue warps read their lanes back (tcgen05.ld), apply
//     a = tanh(z + b) to each node's value column and scale its tangent columns
//     by tanh' = 1 - a^2, and write the next layer's X in place.
// The input layer (17 -> h, tangent = W_0) is computed by the epilogue warps
// in FP32 directly into X; the 3-row output layer is one more MMA (rows padded
// to 128) whose lanes 0..2 are written out as f_D and J_D.
//
// Column order inside a CTA (N dimension of every MMA): node n's first 16
// tangents at columns 16n .. 16n+15, then a tail with all values
// (16 NPC + n) and all 17th tangents (17 NPC + n), padded to a multiple of 16.
// This keeps every tcgen05.ld of 16 columns 16-aligned.
//
// Roles (320 threads): warp 0 issues TMA, warp 1 owns tensor memory and one
// lane issues the MMAs, warps 2..9 are the epilogue (two per TMEM lane
// quadrant, splitting the nodes).  Every mbarrier wait is bounded: on timeout
// the CTA records RTN_E_TIMEOUT in a device flag, stops its pipeline, frees
// its tensor memory and returns.
#include <algorithm>
#include <cstring>

#include "tc_common.cuh"

namespace rtn {
namespace {

// Persistent: CTA b handles node tiles b, b + gridDim.x, ...  The activation
// matrix X is tracked in blocks of 128 rows (one M tile of the producing
// layer = two 64-wide K blocks of the consuming layer), so that
//  * the epilogue of M tile m starts as soon as that tile's accumulator is
//    final, and writes its rows once the current layer's last M tile has read
//    the block it overwrites (xfree, committed inside the MMA stream);
//  * the next layer's MMAs start on every block as soon as it is written
//    (xready), while later blocks are still being produced;
//  * the next tile's input layer is written block by block while the current
//    tile's output layer still runs.
// The producer and the MMA issuer run through the same sequence of
// (tile, layer, M tile, K block) without stopping.
template <int NPC, int MODE, int STAGES>
__global__ void __launch_bounds__(THREADS, 1)
    mlp_tc_kernel(const __grid_constant__ CUtensorMap tmap, TcArgs a) {
  constexpr int C = Cols<NPC>::C, TAIL = Cols<NPC>::TAIL, HALF = (NPC + 1) / 2;
  constexpr int CX = XGeo<C, MODE>::CX;        // columns of one X buffer
  constexpr int NMMA = MODE == 2 ? 2 * C : C;  // N of every MMA = TMEM columns per M tile
  static_assert(NMMA % 16 == 0 && NMMA <= 256, "MMA N");
  constexpr int NZV = NPC * NZ;
  constexpr int MT = 4;  // at most 4 M tiles (hidden width <= 512)
  extern __shared__ uint8_t smem_raw[];
  const int HP = a.HP, nkb = HP / 64, n_mt = HP / 128;
  const int nh = a.n_hidden_mm, n_layers = nh + 1;
  const int n_tiles = (a.n_nodes + NPC - 1) / NPC;
  const uint32_t sraw = smem_u32(smem_raw);
  const uint32_t pad = (1024u - (sraw & 1023u)) & 1023u;
  uint8_t* sm = smem_raw + pad;
  const uint32_t sbase = sraw + pad;
  const uint32_t xbytes = (uint32_t)CX * HP * 2u;  // one X buffer
  const uint32_t xtotal = (MODE == 1 ? 2u : 1u) * xbytes;
  uint8_t* X = sm;
  const uint32_t xhi_s = sbase, xlo_s = sbase + xbytes;
  const uint32_t w_s = sbase + xtotal;
  uint8_t* tail_area = sm + xtotal + STAGES * WT_BYTES;
  const uint32_t bar_s = smem_u32(tail_area);
  auto full_bar = [&](int s) { return bar_s + 8u * s; };
  auto empty_bar = [&](int s) { return bar_s + 8u * (STAGES + s); };
  auto acc_full = [&](int m) { return bar_s + 8u * (2 * STAGES + m); };
  auto tmem_free = [&](int m) { return bar_s + 8u * (2 * STAGES + MT + m); };
  auto xready = [&](int j) { return bar_s + 8u * (2 * STAGES + 2 * MT + j); };
  auto xfree = [&](int j) { return bar_s + 8u * (2 * STAGES + 3 * MT + j); };
  const uint32_t z_full = bar_s + 8u * (2 * STAGES + 4 * MT), z_free = z_full + 8u;
  constexpr int NBAR = 2 * STAGES + 4 * MT + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tail_area + 8 * NBAR);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);
  float* zbuf = reinterpret_cast<float*>(tail_area + 8 * NBAR + 16);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (int m = 0; m < MT; ++m) {
      mbar_init(acc_full(m), 1);
      mbar_init(tmem_free(m), EPI_WARPS);
      mbar_init(xready(m), EPI_WARPS);
      mbar_init(xfree(m), 1);
    }
    mbar_init(z_full, EPI_WARPS);
    mbar_init(z_free, EPI_WARPS);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    // ---------------- TMA producer (whole warp, one elected lane issues)
    if (lane == 0)
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
    {
      int s = 0;
      uint32_t ph = 0;
      bool ok = true;
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x)
        for (int l = 0; l < n_layers && ok; ++l) {
          const int mts = (l < nh) ? n_mt : 1;
          for (int m = 0; m < mts && ok; ++m)
            for (int kb = 0; kb < nkb && ok; ++kb) {
              if (!(ok = mbar_wait_warp(empty_bar(s), ph ^ 1u, abort_flag, a.err))) break;
              if (elect_one()) {
                mbar_expect_tx(full_bar(s), WT_BYTES);
#pragma unroll
                for (int bx = 0; bx < W_BOXES; ++bx)
                  tma_load_2d(w_s + s * WT_BYTES + bx * 4096u, &tmap, kb * 64 + bx * W_BOX_K,
                              l * HP + m * 128, full_bar(s));
              }
              __syncwarp();
              if (++s == STAGES) { s = 0; ph ^= 1u; }
            }
        }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer (whole warp, one elected lane issues)
    {
      constexpr uint32_t idesc = idesc_bf16(128, NMMA) | (1u << 16);  // B is N-major
      const uint32_t lbo = CX * 16u;
      int s = 0;
      uint32_t ph = 0, used = 0, tf_par = 0, xr_par = 0;
      bool ok = true;
      int it = 0;
      WaitClock wc(a.trace != nullptr && blockIdx.x == 0);
      const bool tl = RTN_TRACE && lane == 0;
      for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++it)
        for (int l = 0; l < n_layers && ok; ++l) {
          if (tl) trace(a, it, l, n_layers, 0);
          long long w_x = 0, w_w = 0, w_t = 0;
          const int mts = (l < nh) ? n_mt : 1;
          for (int m = 0; m < mts && ok; ++m) {
            if (used & (1u << m)) {
              wc.start();
              ok = mbar_wait_warp(tmem_free(m), (tf_par >> m) & 1u, abort_flag, a.err);
              wc.stop(w_t);
              if (!ok) break;
              tf_par ^= 1u << m;
            }
            used |= 1u << m;
            tc_fence_after();
            const uint32_t d = tmem + (uint32_t)(m * NMMA);
            for (int kb = 0; kb < nkb && ok; ++kb) {
              const int j = kb >> 1;
              if (m == 0 && (kb & 1) == 0) {
                wc.start();
                ok = mbar_wait_warp(xready(j), (xr_par >> j) & 1u, abort_flag, a.err);
                wc.stop(w_x);
                if (!ok) break;
                xr_par ^= 1u << j;
                tc_fence_after();
              }
              wc.start();
              ok = mbar_wait_warp(full_bar(s), ph, abort_flag, a.err);
              wc.stop(w_w);
              if (!ok) break;
              tc_fence_after();
              const uint32_t as = w_s + s * WT_BYTES;
#pragma unroll
              for (int ks = 0; ks < 4; ++ks) {
                const uint64_t ad = wdesc(as, ks);
                const uint32_t bo = (uint32_t)(kb * 4 + ks) * 2u * lbo;  // 16 k = 2 k-groups
                mma_bf16_elect(d, ad, xdesc(xhi_s + bo, lbo), idesc, (kb | ks) != 0);
                if (MODE == 1) mma_bf16_elect(d, ad, xdesc(xlo_s + bo, lbo), idesc, 1u);
              }
              mma_commit_elect(empty_bar(s));
              if (++s == STAGES) { s = 0; ph ^= 1u; }
              // the last M tile of the layer has read block j: it may be rewritten
              if (m == mts - 1 && (kb & 1)) mma_commit_elect(xfree(j));
            }
            if (ok) mma_commit_elect(acc_full(m));
          }
          if (tl) {
            trace(a, it, l, n_layers, 1);
            trace_put(a, it, l, n_layers, 4, w_x);
            trace_put(a, it, l, n_layers, 5, w_w);
            trace_put(a, it, l, n_layers, 6, w_t);
          }
        }
    }
  } else {
    // ---------------- epilogue warps
    const int e = warp - 2;  // 0..7
    const int q = warp & 3;  // TMEM lane quadrant this warp may access
    const int half = e >> 2;
    const int et = threadIdx.x - 64;  // 0..255
    // zero the X buffers once: pad columns are never written again
    for (uint32_t o = (uint32_t)et * 16u; o < xtotal; o += 256u * 16u)
      *reinterpret_cast<uint4*>(sm + o) = make_uint4(0u, 0u, 0u, 0u);
    float zpref = (et < NZV) ? load_z(a, blockIdx.x * NPC + et / NZ, et % NZ) : 0.0f;
    uint32_t acc_par = 0, xf_par = 0, zf_par = 0, zr_ph = 0;
    bool ok = true, first_input = true;
    const bool tr = RTN_TRACE && (e == 0 && lane == 0);

    // bounded wait by lane 0, result shared with the warp
    long long epi_wait = 0;
    WaitClock ewc(tr && a.trace != nullptr && blockIdx.x == 0);
    auto wwait = [&](uint32_t bar, uint32_t par) -> bool {
      int w_ok = 0;
      ewc.start();
      if (lane == 0) w_ok = mbar_wait(bar, par, abort_flag, a.err);
      ewc.stop(epi_wait);
      return __shfl_sync(0xffffffffu, w_ok, 0) != 0;
    };

    // input layer of tile `tile` (FP32), block by block; thread et handles
    // neuron 128 j + (et % 128) for one half of the nodes
    auto input_layer = [&](int tile, int it_) -> bool {
      const int node0 = tile * NPC;
      if (!wwait(z_free, zr_ph ^ 1u)) return false;  // every warp done with the last z
      zr_ph ^= 1u;
      if (et < NZV) zbuf[et] = zpref;
      __syncwarp();
      if (lane == 0) mbar_arrive(z_full);
      if (!wwait(z_full, zf_par)) return false;
      zf_par ^= 1u;
      if (tr) trace(a, it_, n_layers, n_layers, 0);
      const int hh = et >> 7;
      for (int j = 0; j < n_mt; ++j) {
        if (!first_input) {
          if (!wwait(xfree(j), (xf_par >> j) & 1u)) return false;
          xf_par ^= 1u << j;
        }
        const int i = 128 * j + (et & 127);
        float w[NZ];
#pragma unroll
        for (int jj = 0; jj < NZ; ++jj) w[jj] = a.W0[(size_t)jj * HP + i];
        const float bi = a.b0[i];
#pragma unroll
        for (int n = 0; n < NPC; ++n) {
          if ((n < HALF) != (hh == 0)) continue;
          float s = bi;
#pragma unroll
          for (int jj = 0; jj < NZ; ++jj) s = fmaf(w[jj], zbuf[n * NZ + jj], s);
          const bool real = node0 + n < a.n_nodes;
          const float av = real ? tanh_tc(s) : 0.0f, d = real ? 1.0f - av * av : 0.0f;
          NodeOut o;
          node_pack<MODE>(av, d, w, w[16], o);
          node_store<NPC, C, MODE>(X, xbytes, i, n, o);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) mbar_arrive(xready(j));
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(z_free);
      first_input = false;
      if (tr) trace(a, it_, n_layers, n_layers, 1);
      return true;
    };

    int it = 0;
    if (blockIdx.x < n_tiles) ok = input_layer(blockIdx.x, 0);
    for (int tile = blockIdx.x; tile < n_tiles && ok; tile += gridDim.x, ++it) {
      const int node0 = tile * NPC;
      // hidden layers
      for (int l = 0; l < nh && ok; ++l) {
        for (int m = 0; m < n_mt; ++m) {
          if (!(ok = wwait(acc_full(m), (acc_par >> m) & 1u))) break;
          acc_par ^= 1u << m;
          if (tr && m == 0) trace(a, it, l, n_layers, 2);
          tc_fence_after();
          const int i = 128 * m + 32 * q + lane;
          const float bi = a.bias[(size_t)l * HP + i];
          const uint32_t trow = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(m * NMMA);
          // block m of X may be overwritten once this layer's last M tile read it
          if (!(ok = wwait(xfree(m), (xf_par >> m) & 1u))) break;
          xf_par ^= 1u << m;
          auto store = [&](int n, const NodeOut& o) { node_store<NPC, C, MODE>(X, xbytes, i, n, o); };
          if (half == 0)
            epilogue_nodes<NPC, C, MODE, 0, HALF>(trow, bi, store);
          else
            epilogue_nodes<NPC, C, MODE, HALF, NPC>(trow, bi, store);
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(tmem_free(m));
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          __syncwarp();
          if (lane == 0) mbar_arrive(xready(m));
        }
        if (tr) {
          trace(a, it, l, n_layers, 3);
          trace_put(a, it, l, n_layers, 7, epi_wait);
          epi_wait = 0;
        }
      }
      if (!ok) break;
      // next tile's input layer, overlapping this tile's output layer
      const int nt = tile + gridDim.x;
      if (nt < n_tiles) {
        if (et < NZV) zpref = load_z(a, nt * NPC + et / NZ, et % NZ);
        if (!(ok = input_layer(nt, it + 1))) break;
      }
      // output layer: TMEM lanes 0..2 of M tile 0 hold the three outputs
      if (!(ok = wwait(acc_full(0), acc_par & 1u))) break;
      acc_par ^= 1u;
      if (tr) trace(a, it, nh, n_layers, 2);
      tc_fence_after();
      if (q == 0) {
        float tl[TAIL];
#pragma unroll
        for (int c = 0; c < TAIL / 16; ++c) tmem_ld16_sum<C, MODE>(tmem + 16 * NPC + 16 * c, tl + 16 * c);
        tmem_wait_ld();
        const float bo = lane < NO ? a.bias[(size_t)nh * HP + lane] : 0.0f;
#pragma unroll
        for (int n = 0; n < NPC; ++n) {
          if ((n < HALF) != (half == 0)) continue;
          float t[16];
          tmem_ld16_sum<C, MODE>(tmem + 16 * n, t);
          tmem_wait_ld();
          const int node = node0 + n;
          if (lane < NO && node < a.n_nodes) {
            a.fD[(size_t)node * NO + lane] = tl[n] + bo;
            float* J = a.JD + (size_t)node * NO * NZ + lane * NZ;
#pragma unroll
            for (int j = 0; j < 16; ++j) J[j] = t[j];
            J[16] = tl[NPC + n];
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tmem_free(0));
    }
  }

  __syncthreads();
  if (warp == 1) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(a.tmem_cols)
                 : "memory");
  }
}

// ---------------------------------------------------------------- host side

struct Variant {
  int npc;
  int mode;  // 0 single, 1 split (two MMAs), 2 split (hi|lo along N), (3: the forward mode
             // on CTA pairs, no longer compiled: it won no shape / batch size),
             // 4 split, reverse mode (value forward, three adjoints backward),
             // 5 split, reverse mode on a CTA pair,
             // 6 split, reverse mode layered (one GEMM per layer over all nodes),
             // 7 as 6 with the hidden forward and backward GEMMs on CTA
             //   pairs (hidden width a multiple of 256)
  int stages;
  const void* fn;
  bool split() const { return mode != 0; }
  bool pair() const { return mode == 5; }
  bool rev() const { return mode == 4 || mode == 5; }
  bool layered() const { return mode == 6 || mode == 7; }
  int threads() const { return pair() ? THREADS + 32 : THREADS; }
  int cols() const { return rev() ? 128 : 16 * npc + ((2 * npc + 15) / 16) * 16; }
  // tensor-memory columns of one accumulator tile (128 rows; 256 rows on a pair)
  int tmem_per_mtile() const { return mode == 5 ? 256 : rev() ? 128 : (mode >= 2 ? 2 * cols() : cols()); }
  int rows_per_mtile() const { return (pair() || mode == 7) ? 256 : 128; }
  // accumulator columns: one slot per M tile (a pair always has two slots:
  // its output layer accumulates in the second)
  int tmem_columns(int HP) const {
    return (pair() ? std::max(2, HP / 256) : HP / 128) * tmem_per_mtile();
  }
  size_t smem(int HP) const {
    if (layered()) return mlp_lay_smem();
    if (mode == 5) return mlp_rev2_smem(HP, stages);
    if (rev())
      return 1024 + (size_t)128 * HP * 2 + (size_t)stages * WT_BYTES + 8 * (2 * stages + 20) + 16 +
             (size_t)npc * ZS * 4;
    return 1024 + (mode != 0 ? 2 : 1) * (size_t)cols() * HP * 2 + (size_t)stages * WT_BYTES +
           8 * (2 * stages + 18) + 16 + (size_t)npc * NZ * 4;
  }
};

template <int NPC, int MODE, int STAGES>
Variant variant() {
  return Variant{NPC, MODE, STAGES, (const void*)&mlp_tc_kernel<NPC, MODE, STAGES>};
}

template <int NPC, int STAGES>
Variant rev_variant() {
  return Variant{NPC, 4, STAGES, mlp_rev_fn(NPC, STAGES)};
}

template <int STAGES>
Variant rev2_variant() {
  return Variant{42, 5, STAGES, mlp_rev2_fn(42, STAGES)};
}

Variant lay_variant(int mode) { return Variant{0, mode, 2, mlp_lay_fn()}; }

// every compiled tile shape; the autotuner times those that fit
const std::vector<Variant>& all_variants() {
  static const std::vector<Variant> v = {
      variant<14, 0, 6>(), variant<14, 0, 5>(), variant<8, 0, 8>(), variant<7, 0, 5>(),
      variant<6, 0, 6>(),  variant<4, 0, 8>(),  variant<8, 1, 4>(),
      variant<5, 1, 6>(),  variant<4, 1, 3>(),  variant<3, 1, 6>(),  variant<7, 2, 5>(),
      variant<7, 2, 8>(),  variant<4, 2, 6>(),  variant<3, 2, 5>(),  rev_variant<21, 6>(),
      rev_variant<21, 4>(), rev_variant<16, 6>(), rev2_variant<3>(), rev2_variant<6>(), lay_variant(6),
      lay_variant(7)};
  return v;
}

bool fits(const Variant& v, int HP) {
  if (!v.fn || HP % v.rows_per_mtile() != 0) return false;
  return v.smem(HP) <= 232448 && v.tmem_columns(HP) <= 512;
}

// default before autotuning: with split operands the reverse-mode tile (the
// fewest MMAs per node; on CTA pairs from hidden width 512, where a single
// CTA's MMAs are bound by shared-memory bytes); otherwise the widest tile that
// still leaves >= 3 stages
int default_variant(int HP, bool split) {
  const auto& vs = all_variants();
  int best = -1;
  for (int i = 0; i < (int)vs.size(); ++i) {
    if (vs[i].split() != split || !fits(vs[i], HP) || vs[i].stages < 3) continue;
    // reverse mode first, then the widest MMA (fewest instructions per
    // column), then one CTA before a pair, then the most columns
    auto key = [&](const Variant& v) {
      const int rank = v.mode == 5 ? (HP >= 512 ? 3 : 1) : v.mode == 4 ? 2 : 0;
      return rank * 100000000 + v.tmem_per_mtile() * 10000 + (v.pair() ? 0 : 5000) + v.cols() * 10 + v.npc;
    };
    if (best < 0 || key(vs[i]) > key(vs[best])) best = i;
  }
  return best;
}

// the layered reverse-mode shapes are the only ones of RTN_FP8; the default
// runs its hidden GEMMs on single CTAs (tile mode 6).  On CTA pairs (mode 7,
// selectable) the FP8 GEMMs measured slower at the precision workload
// (backward 0.594 vs 0.535 ms, forward 0.186 vs 0.163 ms per launch): their
// epilogues, not the operand traffic the pairs halve, bound them, and a pair
// frees an accumulator only when both CTAs' epilogues are done.
int layered_variant(int HP) {
  const auto& vs = all_variants();
  for (int i = 0; i < (int)vs.size(); ++i)
    if (vs[i].mode == 6 && fits(vs[i], HP)) return i;
  return -1;
}

uint16_t f2bf(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7fffffffu) > 0x7f800000u) return 0x7fc0;
  u += 0x7fffu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}

cudaError_t select_variant(rtn_ctx* ctx, int idx) {
  TcNet& tc = ctx->net.tc;
  const Variant& v = all_variants()[idx];
  tc.variant = idx;
  tc.cols = v.cols();
  tc.npc = v.npc;
  tc.stages = v.stages;
  tc.smem = v.smem(tc.h_pad);
  tc.fn = v.fn;
  int ncol = 32;
  while (ncol < v.tmem_columns(tc.h_pad)) ncol *= 2;
  tc.tmem_cols = ncol;
  if (v.layered()) {  // buffers and maps of the layered path (once)
    std::string e;
    cudaError_t ce = mlp_lay_prepare(ctx, e);
    if (ce != cudaSuccess) return ce;
    if (!e.empty()) return cudaErrorNotSupported;
    mlp_lay_set_pair(ctx, v.mode == 7);
    return cudaSuccess;
  }
  return cudaFuncSetAttribute(tc.fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)tc.smem);
}

}  // namespace

cudaError_t mlp_tc_prepare(rtn_ctx* ctx, std::string& err) {
  Net& net = ctx->net;
  TcNet& tc = net.tc;
  const int L = net.n_layers;
  int hmax = 0;
  for (int l = 1; l < L; ++l) hmax = std::max(hmax, net.widths[l]);
  if (hmax > 512) {
    err = "tensor-core path supports hidden widths <= 512";
    return cudaSuccess;
  }
  const int HP = ((hmax + 127) / 128) * 128;
  const int nh = L - 2;  // hidden -> hidden layers on the tensor cores
  tc.h_pad = HP;
  tc.n_mm = nh;
  tc.rows_total = nh * HP + 256;  // output layer padded to one 256-row pair tile
  const bool split = ctx->opt.precision != RTN_BF16;
  const int vi = ctx->opt.precision == RTN_FP8 ? layered_variant(HP) : default_variant(HP, split);
  if (vi < 0) {
    err = "no tensor-core tile configuration fits";
    return cudaSuccess;
  }
  {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&tc.n_sm, cudaDevAttrMultiProcessorCount, dev);
  }

  // host copies of the network (FP32 as given at create)
  std::vector<float> hW, hb;
  {
    size_t nw = 0, nb = 0;
    for (int l = 0; l < L; ++l) {
      nw += (size_t)net.widths[l + 1] * net.widths[l];
      nb += net.widths[l + 1];
    }
    hW.resize(nw);
    hb.resize(nb);
    cudaError_t e = cudaMemcpy(hW.data(), net.W32, nw * 4, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(hb.data(), net.b32, nb * 4, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return e;
  }
  std::vector<uint16_t> Wp((size_t)tc.rows_total * HP, 0);
  std::vector<float> bias((size_t)nh * HP + 128, 0.0f), W0((size_t)HP * NZ, 0.0f), b0(HP, 0.0f);
  for (int l = 0; l < L; ++l) {
    const int fi = net.widths[l], fo = net.widths[l + 1];
    const float* Wl = hW.data() + net.w_off[l];
    const float* bl = hb.data() + net.b_off[l];
    if (l == 0) {
      for (int i = 0; i < fo; ++i) {
        for (int j = 0; j < NZ; ++j) W0[(size_t)j * HP + i] = Wl[(size_t)i * fi + j];
        b0[i] = bl[i];
      }
    } else {
      const size_t row0 = (size_t)(l - 1) * HP;
      for (int i = 0; i < fo; ++i) {
        for (int k = 0; k < fi; ++k) Wp[(row0 + i) * HP + k] = f2bf(Wl[(size_t)i * fi + k]);
        bias[row0 + i] = bl[i];
      }
    }
  }
  // reverse mode (mlp_rev.cu): the same rows, then the transposes of the
  // hidden layers, then W_0' as BF16 hi and lo rows; the output layer in FP32
  const size_t tb = (size_t)nh * HP + 128, rows_r = tb + (size_t)nh * HP + 256;
  std::vector<uint16_t> WRh(rows_r * HP, 0);
  std::copy(Wp.begin(), Wp.begin() + tb * HP, WRh.begin());
  std::vector<float> WL((size_t)NO * HP, 0.0f);
  for (int l = 1; l < L; ++l) {
    const int fi = net.widths[l], fo = net.widths[l + 1];
    const float* Wl = hW.data() + net.w_off[l];
    if (l < L - 1) {
      const size_t row0 = tb + (size_t)(l - 1) * HP;
      for (int i = 0; i < fi; ++i)
        for (int k = 0; k < fo; ++k) WRh[(row0 + i) * HP + k] = f2bf(Wl[(size_t)k * fi + i]);
    } else {
      for (int i = 0; i < NO; ++i)
        for (int k = 0; k < fi; ++k) WL[(size_t)i * HP + k] = Wl[(size_t)i * fi + k];
    }
  }
  {
    const int fo = net.widths[1];
    const float* W0l = hW.data() + net.w_off[0];
    for (int j = 0; j < NZ; ++j)
      for (int k = 0; k < fo; ++k) {
        const float w = W0l[(size_t)k * NZ + j];
        const uint16_t h = f2bf(w);
        const uint32_t hb = (uint32_t)h << 16;
        float hf;
        memcpy(&hf, &hb, 4);
        WRh[(tb + (size_t)nh * HP + j) * HP + k] = h;
        WRh[(tb + (size_t)nh * HP + 128 + j) * HP + k] = f2bf(w - hf);
      }
  }
  cudaError_t e = cudaMalloc(&tc.W, Wp.size() * 2);
  if (e == cudaSuccess) e = cudaMemcpy(tc.W, Wp.data(), Wp.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&tc.WR, WRh.size() * 2);
  if (e == cudaSuccess) e = cudaMemcpy(tc.WR, WRh.data(), WRh.size() * 2, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&tc.WL32, WL.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(tc.WL32, WL.data(), WL.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMalloc(&tc.dscr, (size_t)std::max(1, tc.n_sm) * (nh + 1) * HP * REV_NPC_MAX * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&tc.bias, bias.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(tc.bias, bias.data(), bias.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&tc.W0, W0.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(tc.W0, W0.data(), W0.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&tc.b0, b0.size() * 4);
  if (e == cudaSuccess) e = cudaMemcpy(tc.b0, b0.data(), b0.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMalloc(&tc.err, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(tc.err, 0, sizeof(int));
  if (e != cudaSuccess) return e;

  // tensor map over the stacked BF16 weights: inner dim K = HP, outer = rows
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult qr;
  e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr);
  if (e != cudaSuccess || !fn || qr != cudaDriverEntryPointSuccess) {
    err = "cuTensorMapEncodeTiled unavailable";
    return cudaSuccess;
  }
  auto encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  cuuint64_t dims[2] = {(cuuint64_t)HP, (cuuint64_t)tc.rows_total};
  cuuint64_t strides[1] = {(cuuint64_t)HP * 2};
  cuuint32_t box[2] = {(cuuint32_t)W_BOX_K, 128};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = encode(reinterpret_cast<CUtensorMap*>(tc.tmap_bytes), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                      tc.W, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                      CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return cudaSuccess;
  }
  cuuint64_t dimsR[2] = {(cuuint64_t)HP, (cuuint64_t)rows_r};
  r = encode(reinterpret_cast<CUtensorMap*>(tc.tmapR_bytes), CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, tc.WR,
             dimsR, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return cudaSuccess;
  }
  return select_variant(ctx, vi);
}

cudaError_t mlp_tc_forward(rtn_ctx* ctx, const float* x, const float* u, float* fD, float* JD) {
  TcNet& tc = ctx->net.tc;
  TcArgs a;
  a.x = x;
  a.u = u;
  a.node_inst = ctx->lay.node_inst;
  a.n_nodes = ctx->lay.n_nodes;
  a.W0 = tc.W0;
  a.b0 = tc.b0;
  a.bias = tc.bias;
  a.HP = tc.h_pad;
  a.n_hidden_mm = tc.n_mm;
  a.tmem_cols = (uint32_t)tc.tmem_cols;
  a.fD = fD;
  a.JD = JD;
  a.err = tc.err;
  a.trace = tc.trace;
  const CUtensorMap* map = reinterpret_cast<const CUtensorMap*>(tc.tmap_bytes);
  void* args[] = {(void*)map, (void*)&a};
  const int n_tiles = (a.n_nodes + tc.npc - 1) / tc.npc;
  const Variant& v = all_variants()[tc.variant];
  if (v.layered()) return mlp_lay_launch(ctx, x, u, fD, JD);
  if (v.mode == 5) return mlp_rev2_launch(ctx, x, u, fD, JD);
  if (v.rev()) return mlp_rev_launch(ctx, x, u, fD, JD);
  const dim3 grid(std::min(n_tiles, std::max(1, tc.n_sm)));
  return cudaLaunchKernel(tc.fn, grid, dim3(v.threads()), args, tc.smem, ctx->stream);
}

int mlp_tc_variant_count() { return (int)all_variants().size(); }

// describe variant idx: returns 0 if it fits this network, writes its shape
int mlp_tc_variant_info(rtn_ctx* ctx, int idx, int* npc, int* split, int* stages) {
  const auto& vs = all_variants();
  if (idx < 0 || idx >= (int)vs.size()) return -1;
  if (npc) *npc = vs[idx].npc;
  if (split) *split = vs[idx].mode;
  if (stages) *stages = vs[idx].stages;
  const bool want = ctx->opt.precision != RTN_BF16;
  if (ctx->opt.precision == RTN_FP8 && !vs[idx].layered()) return 1;  // FP8: layered tiles only
  return (vs[idx].split() == want && fits(vs[idx], ctx->net.tc.h_pad)) ? 0 : 1;
}

cudaError_t mlp_tc_select(rtn_ctx* ctx, int idx) { return select_variant(ctx, idx); }

void mlp_tc_release(rtn_ctx* ctx) {
  mlp_lay_release(ctx);
  TcNet& tc = ctx->net.tc;
  void* ptrs[] = {tc.W, tc.bias, tc.W0, tc.b0, tc.err, tc.trace, tc.WR, tc.WL32, tc.dscr};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  tc = TcNet{};
}

int mlp_tc_take_error(rtn_ctx* ctx) {
  TcNet& tc = ctx->net.tc;
  if (!tc.err) return 0;
  int v = 0;
  cudaMemcpy(&v, tc.err, sizeof(int), cudaMemcpyDeviceToHost);
  if (v) cudaMemset(tc.err, 0, sizeof(int));
  return v;
}

}  // namespace rtn
