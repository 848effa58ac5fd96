// Batched form for images too large for one SM (N in {256, 512, 1024}): every image of a size class (or
// of a chunk of it) is one field of a single persistent cooperative launch.
//
// One launch of a single large image leaves most of the GPU idle (a 512 x 512 field has only 16 row and
// 16 column work items per phase) and pays two grid barriers per sweep for very little work. Here all
// fields advance together, sweep by sweep: a row phase over every (field, row block) and a column phase
// over every (field, column block), separated by the same bounded grid barrier as k_global. Each field
// runs its own schedule (Alg. 1 with A = I): the lambda-cooled Wiener solve of §2.2 from s = 0, then,
// from s_W, n_samples sweeps of the sampler; fields that finish early drop out of the work lists.
//
// Per-field schedule state is double-buffered by sweep parity: during the row phase of sweep s every CTA
// that owns a row block of field f reads state[s & 1][f] and the residual sums of the previous column
// phase, derives the same new state, and the owner of row block 0 stores it in state[(s + 1) & 1][f],
// which the column phase of sweep s reads after the barrier.
#pragma once

#include "wf_batch.cuh"
#include "wf_global.cuh"

namespace wf {

// one image of a large-image batch launch (device array, filled on the host)
struct GBField {
  const float2* aq;   // [W][H] sampler pixel table (a, q)
  const float2* dn;   // [W][H] Wiener-filter pixel table (d, 1/N_bar)
  const float2* fg;   // [H][W/2+1] sampler mode table
  const float* Pk;    // [H][W/2+1]
  float2* Z;          // [H][W/2] packed half spectrum (state)
  float2* prev;       // [H][W/2] previous Wiener iterate for the residual
  float* out_wf;      // [H][W] or null
  float* out_samples; // [n_samples][H][W] or null
  uint32_t chain, key0, key1;
  int item;           // index of the batch result
};

// per-field schedule (64 bytes, read with 16-byte L2 loads)
struct __align__(16) GBState {
  double lam, rho;
  float ltau;
  int phase;      // 0 Wiener solve, 1 sampling, 2 finished
  int lev, k, it; // cooling level, sweeps at this level, solve sweeps
  int parity;     // residual accumulator in use
  int status;     // solve status (1 while running)
  int cmp, store; // residual bookkeeping of this sweep's column phase
  int d;          // sampler step word of this sweep
};
static_assert(sizeof(GBState) == 64, "GBState layout");

struct GBArgs {
  const GBField* fields;
  const Scalars* sc;   // [F] per-field set-up
  GBState* state;      // [2][F]
  double* acc;         // [F][2] residual sums
  double* bnorm;       // [F][kMaxLevels] ||S N_lambda^-1 d||^2 per level
  BatchResult* res;    // indexed by GBField::item
  int* active;         // fields not finished (starts at F)
  GridBar* bar;
  const float2* tw_row;
  const float2* tw_col;
  const float2* tw_real;
  int F;
  double tol, eta, level_tol;
  int max_iter, level_max, check, n_samples;
  int grid_pct;        // host side: percent of the co-resident grid
};

__device__ __forceinline__ GBState gb_load(const GBState* p) {
  GBState s;
  const int4* src = reinterpret_cast<const int4*>(p);
  int4* dst = reinterpret_cast<int4*>(&s);
#pragma unroll
  for (int i = 0; i < 4; ++i) dst[i] = __ldcg(src + i);
  return s;
}

__device__ __forceinline__ int block_max_levels(const Scalars* sc, int F, int* red) {
  int m = 0;
  for (int f = threadIdx.x; f < F; f += 128) {
    const Scalars s = sc[f];
    if (s.status == 0 && s.n_levels > m) m = s.n_levels;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  const int r = max(max(red[0], red[1]), max(red[2], red[3]));
  __syncthreads();
  return r;
}

// rows y0 .. y0+RB-1 of field Z: load and inverse row transform (C2R) into buf, or zeros
template <int N>
__device__ __forceinline__ void gb_rows_in(const GBArgs& a, float2* buf, const float2* Z, int y0, bool zero) {
  using G = GGeo<N>;
  constexpr int L = G::LR;
  if (zero) {
    for (int e = threadIdx.x; e < G::RB * L; e += 128) buf[(e / L) * G::VROW + padi(e % L)] = make_float2(0.f, 0.f);
    __syncthreads();
    return;
  }
  for (int e = threadIdx.x; e < G::RB * L; e += 128) {
    const int j = e / L, m = e % L;
    buf[j * G::VROW + padi(m)] = __ldcg(Z + (long long)(y0 + j) * L + m);
  }
  __syncthreads();
  real_pass<N, false>(buf, G::RB, a.tw_real);
  fft_smem<G::RR, G::RB, G::VROW, true, G::SR>(buf, a.tw_row);
}

// the real rows in buf to out[y0 .. y0+RB-1][W]
template <int N>
__device__ __forceinline__ void gb_rows_emit(const float2* buf, float* out, int y0) {
  using G = GGeo<N>;
  constexpr int L = G::LR;
  for (int e = threadIdx.x; e < G::RB * L; e += 128) {
    const int j = e / L, m = e % L;
    reinterpret_cast<float2*>(out + (long long)(y0 + j) * G::W)[m] = buf[j * G::VROW + padi(m)];
  }
}

// forward row transform (R2C) of buf and store into Z
template <int N>
__device__ __forceinline__ void gb_rows_out(const GBArgs& a, float2* buf, float2* Z, int y0) {
  using G = GGeo<N>;
  constexpr int L = G::LR;
  fft_smem<G::RR, G::RB, G::VROW, false, G::SR>(buf, a.tw_row);
  real_pass<N, true>(buf, G::RB, a.tw_real);
  for (int e = threadIdx.x; e < G::RB * L; e += 128) {
    const int j = e / L, m = e % L;
    __stcg(Z + (long long)(y0 + j) * L + m, buf[j * G::VROW + padi(m)]);
  }
  __syncthreads();
}

// column item: load, forward column FFT, spectral update, and (mode != 2) inverse FFT and store
template <int N>
__device__ __forceinline__ double gb_cols(const GBArgs& a, float2* buf, const GBField& fd, int c0, int mode,
                                          uint32_t step, float ltau, bool cmp, bool store) {
  using G = GGeo<N>;
  constexpr int L = G::LR, H = G::H;
  for (int e = threadIdx.x; e < G::CB * H; e += 128) {
    const int j = e % G::CB, y = e / G::CB;
    buf[j * G::VCOL + padi(y)] = __ldcg(fd.Z + (long long)y * L + c0 + j);
  }
  __syncthreads();
  fft_smem<G::RC, G::CB, G::VCOL, false, G::SC>(buf, a.tw_col);
  const double acc =
      col_update<N>(mode, buf, c0, fd.fg, fd.Pk, fd.prev, step, fd.chain, fd.key0, fd.key1, ltau, cmp, store);
  if (mode == 2) return acc;
  fft_smem<G::RC, G::CB, G::VCOL, true, G::SC>(buf, a.tw_col);
  for (int e = threadIdx.x; e < G::CB * H; e += 128) {
    const int j = e % G::CB, y = e / G::CB;
    __stcg(fd.Z + (long long)y * L + c0 + j, buf[j * G::VCOL + padi(y)]);
  }
  __syncthreads();
  return acc;
}

template <int N>
__global__ void __launch_bounds__(128, 3) k_gbatch(GBArgs a) {
  using G = GGeo<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float2* buf = reinterpret_cast<float2*>(smem_raw);
  __shared__ double red[4];
  __shared__ int ired[4];
  constexpr double NPIX = double(G::H * G::W);
  const unsigned int nb = gridDim.x;
  const int F = a.F;
  const int row_items = G::ROW_ITEMS * F, col_items = G::COL_ITEMS * F;

  // 1. level norms, one cooling level at a time for all fields
  const int max_levels = block_max_levels(a.sc, F, ired);
  for (int l = 0; l < max_levels; ++l) {
    for (int it = blockIdx.x; it < row_items; it += nb) {
      const int f = it / G::ROW_ITEMS, y0 = (it % G::ROW_ITEMS) * G::RB;
      const Scalars sc = a.sc[f];
      if (sc.status != 0 || l >= sc.n_levels) continue;
      const GBField fd = a.fields[f];
      gb_rows_in<N>(a, buf, fd.Z, y0, true);
      pixel_update<N>(2, buf, y0, fd.aq, fd.dn, 0u, 0u, 0u, 0u, 0.f, 0.f, 0,
                      float(level_lambda(sc, l, a.eta) * sc.tau));
      gb_rows_out<N>(a, buf, fd.Z, y0);
    }
    if (!grid_barrier(a.bar, nb)) return;
    for (int it = blockIdx.x; it < col_items; it += nb) {
      const int f = it / G::COL_ITEMS;
      const Scalars sc = a.sc[f];
      if (sc.status != 0 || l >= sc.n_levels) continue;
      const GBField fd = a.fields[f];
      const double s = block_sum_128(gb_cols<N>(a, buf, fd, (it % G::COL_ITEMS) * G::CB, 2, 0u, 0.f, false, false), red);
      if (threadIdx.x == 0) atomicAdd(a.bnorm + f * kMaxLevels + l, s / NPIX);
    }
    if (!grid_barrier(a.bar, nb)) return;
  }

  // 2. sweeps: every field's Wiener solve, then its samples from s_W
  const long long max_sweeps = (long long)a.max_iter + a.n_samples + 4;
  for (long long sw = 0; sw < max_sweeps; ++sw) {
    const GBState* cur = a.state + (sw & 1) * F;
    GBState* nxt = a.state + ((sw + 1) & 1) * F;
    for (int it = blockIdx.x; it < row_items; it += nb) {
      const int f = it / G::ROW_ITEMS, rb = it % G::ROW_ITEMS, y0 = rb * G::RB;
      const bool owner = rb == 0 && threadIdx.x == 0;
      const Scalars sc = a.sc[f];
      const GBField fd = a.fields[f];
      GBState S;
      const bool fresh = sw == 0;
      if (fresh) {
        S.lam = sc.lam0;
        S.rho = -1.0;
        S.ltau = float(sc.lam0 * sc.tau);
        S.phase = 0;
        S.lev = S.k = S.it = S.parity = 0;
        S.status = 1;
        S.cmp = S.store = 0;
        S.d = 0;
        if (sc.status != 0) {  // set-up failed: no solve, no samples
          S.phase = 2;
          S.status = sc.status;
          if (owner) {
            a.res[fd.item] = BatchResult{-1.0, 0, sc.status};
            nxt[f] = S;
            atomicSub(a.active, 1);
          }
          continue;
        }
      } else {
        S = gb_load(cur + f);
        if (S.phase == 2) {
          if (owner) nxt[f] = S;
          continue;
        }
      }
      // decisions on the previous column phase (as in k_global's schedule)
      if (!fresh && S.phase == 0) {
        if (S.cmp) {
          const double tot = __ldcg(a.acc + 2 * f + S.parity) * NPIX;
          if (owner) a.acc[2 * f + (S.parity ^ 1)] = 0.0;  // the next check's accumulator
          S.parity ^= 1;
          const double bn = __ldcg(a.bnorm + f * kMaxLevels + S.lev);
          const double r2 = bn > 0.0 ? tot / bn : tot;
          S.rho = sqrt(r2);
          if (!(r2 == r2) || r2 > 1e300) {
            S.status = 6;
          } else if (S.lev < sc.n_levels - 1) {
            if (S.rho < a.level_tol || S.k >= a.level_max) {
              ++S.lev;
              S.lam = level_lambda(sc, S.lev, a.eta);
              S.ltau = float(S.lam * sc.tau);
              S.k = 0;
            }
          } else if (S.rho < a.tol) {
            S.status = 0;
          }
        }
        if (S.status == 1 && S.it >= a.max_iter) S.status = 5;
      }
      gb_rows_in<N>(a, buf, fd.Z, y0, fresh);
      bool finished = false;
      if (S.phase == 0 && S.status != 1) {  // solve done: s_W out, then samples from it
        if (fd.out_wf) gb_rows_emit<N>(buf, fd.out_wf, y0);
        if (owner) a.res[fd.item] = BatchResult{S.rho, S.it, S.status};
        if (a.n_samples > 0 && fd.out_samples) {
          S.phase = 1;
          S.d = 0;
        } else {
          finished = true;
        }
      } else if (S.phase == 1) {  // the sweep with step word d is complete: sample d
        gb_rows_emit<N>(buf, fd.out_samples + (long long)S.d * (G::H * G::W), y0);
        ++S.d;
        finished = S.d >= a.n_samples;
      }
      __syncthreads();  // emitted rows are read above with another thread mapping than the update below
      if (finished) {
        S.phase = 2;
        if (owner) {
          nxt[f] = S;
          atomicSub(a.active, 1);
        }
        continue;
      }
      if (S.phase == 0) {
        ++S.k;
        ++S.it;
        S.cmp = (S.k % a.check == 0) && S.k >= 2;
        S.store = ((S.k + 1) % a.check == 0);
        pixel_update<N>(1, buf, y0, fd.aq, fd.dn, 0u, 0u, 0u, 0u, 0.f, S.ltau, 0, 0.f);
      } else {
        pixel_update<N>(0, buf, y0, fd.aq, fd.dn, uint32_t(S.d), fd.chain, fd.key0, fd.key1, sc.sqrt_tau, 0.f, 0,
                        0.f);
      }
      gb_rows_out<N>(a, buf, fd.Z, y0);
      if (owner) nxt[f] = S;
    }
    if (!grid_barrier(a.bar, nb)) return;
    // no field changes state between here and the next barrier: every CTA sees the same count
    if (__ldcg(a.active) == 0) return;
    for (int it = blockIdx.x; it < col_items; it += nb) {
      const int f = it / G::COL_ITEMS;
      const GBState S = gb_load(nxt + f);
      if (S.phase == 2) continue;
      const GBField fd = a.fields[f];
      const int c0 = (it % G::COL_ITEMS) * G::CB;
      if (S.phase == 0) {
        const double part = block_sum_128(gb_cols<N>(a, buf, fd, c0, 1, 0u, S.ltau, S.cmp != 0, S.store != 0), red);
        if (S.cmp && threadIdx.x == 0) atomicAdd(a.acc + 2 * f + S.parity, part);
      } else {
        gb_cols<N>(a, buf, fd, c0, 0, uint32_t(S.d), 0.f, false, false);
      }
    }
    if (!grid_barrier(a.bar, nb)) return;
  }
}

}  // namespace wf
