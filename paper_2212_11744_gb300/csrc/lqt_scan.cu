// Stages (b) and (c): the reverse scan of the elements with the LQT
// combination (Sec. III-D Theorem parallel_HJB, Sec. IV-A eq. lqt_comb) and the
// forward scan of the one-sub-interval affine maps of the optimal state
// (Sec. IV-E, Method 1 combination eqs. Psi_comb/alpha_comb).
//
// Both scans are chunked and hierarchical instead of a Blelloch up/down sweep
// over single elements:
//   level 0: each thread owns a chunk of G0 consecutive elements;
//   reduce : each thread folds its group (right to left) into one aggregate,
//            giving the next level's elements;
//   top    : one group left -> fold it sequentially from the zero value;
//   down   : each thread re-folds its group in VALUE form, starting from the
//            suffix value of everything to its right (read from the level
//            above).  A value-form combination costs about 40% of a full one
//            and yields the optimal-state map of that sub-interval for free.
// Level 0 uses long chunks (the wide level, throughput-bound); upper levels
// use pairs (they are latency-bound: on this GPU one FP64 warp instruction
// occupies a sub-partition for ~62 cycles whatever the lane count, so the
// critical path is what counts there).
#include <cuda_runtime.h>

#include "lqt_device.cuh"
#include "lqt_internal.h"

namespace lqt {

constexpr int kUpperGroup = 2;

static thread_local int t_chunk_override = 0;
void set_scan_chunk(int g) { t_chunk_override = g; }
int scan_chunk_override() { return t_chunk_override; }

// Level-0 chunk length from T, or the caller's override.  Level 0 is FP64
// throughput-bound with one thread per chunk, and a sub-partition runs one
// FP64 warp instruction per 64 cycles whatever its warp count, so the chunks
// are sized to give every one of the 152 x 4 sub-partitions the same number of
// warps -- two, so that one warp's memory and dependency stalls are covered by
// the other (152 * 4 * 32 * 2 = 38912 threads); an uneven count would leave
// some sub-partitions with one warp more than others at the end.  At least 2,
// at most 64 elements per chunk.
constexpr int64_t kLevel0Threads = 152 * 4 * 32 * 2;
static int level0_group(int64_t T) {
  if (t_chunk_override >= 2) return t_chunk_override;
  int64_t g = (T + 1 + kLevel0Threads - 1) / kLevel0Threads;
  if (g < 2) g = 2;
  if (g > 64) g = 64;
  return (int)g;
}

static int64_t ceil_div(int64_t a, int64_t b) { return (a + b - 1) / b; }

static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

// ---------------------------------------------------------------------------
// element source: the public SoA arrays (level 0)
// ---------------------------------------------------------------------------

template <int N>
struct SrcPublic {
  ElemPtrs el;
  __device__ __forceinline__ void load(int64_t k, Elem<N>& e) const { load_public<N>(el, k, e); }
};
// full-matrix records of the upper levels (full_elem_doubles layout)
template <int N>
struct SrcFull {
  const double* p;
  __device__ __forceinline__ void load(int64_t k, Elem<N>& e) const { load_full<N>(p + k * full_elem_doubles<N>(), e); }
};

// ---------------------------------------------------------------------------
// value scan kernels
// ---------------------------------------------------------------------------

// agg[g] = e[gG] (x) e[gG+1] (x) ... (x) e[min(gG+G, cnt)-1], stored as a
// full-matrix record for the warp-per-combination upper levels.
template <int N, class Src, typename GT = double>
__global__ void __launch_bounds__(128) reduce_elems_kernel(Src src, int64_t cnt, int G, double* __restrict__ agg) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t first = g * G;
  if (first >= cnt) return;
  const int64_t last = (first + G < cnt ? first + G : cnt) - 1;
  Elem<N> acc, e;
  src.load(last, acc);
  for (int64_t k = last - 1; k >= first; --k) {
    src.load(k, e);
    combine<N, GT>(e, acc, acc);
  }
  store_full<N>(agg + g * full_elem_doubles<N>(), acc);
}

struct DownOut {
  // level-0 outputs (public layout); zeta may be null
  double *S, *v, *zeta;
  // level-0 optimal-state maps and chunk composites (may be null)
  double* maps;       // [T][N*N + N]
  double* composite;  // [chunks-1][N*N + N]
  int64_t T;
  // batches: zeta[k] receives the element's own share of zeta (zeta_k minus
  // zeta_{k+1}, formed without that subtraction); a segmented suffix sum per
  // problem then gives zeta without the later problems' zeta leaking in
  int zeta_inc;
};

template <int N>
__device__ __forceinline__ void store_val_public(const DownOut& o, int64_t k, const Val<N>& V) {
  double* S = o.S + k * N * N;
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = 0; j < N; ++j) S[i * N + j] = V.S[sidx<N>(i, j)];
#pragma unroll
  for (int i = 0; i < N; ++i) o.v[k * N + i] = V.v[i];
  if (o.zeta) o.zeta[k] = V.zeta;
  bool ok = isfinite(V.zeta);
#pragma unroll
  for (int i = 0; i < Dim<N>::NS; ++i) ok = ok && isfinite(V.S[i]);
  if (!ok) flag(kStatusNonFinite);
}

// Suffix values of one level-0 group, right to left, from the carry `above`
// (the value of everything after the group, a full-matrix value record; zero
// value at the right end), with the one-sub-interval optimal-state maps and
// the chunk's composite map.
template <int N, class Src, typename GT = double>
__global__ void __launch_bounds__(128) down_values_kernel(Src src, int64_t cnt, int G, const double* __restrict__ above,
                                                          int64_t cnt_above, DownOut o) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t first = g * G;
  if (first >= cnt) return;
  const int64_t last = (first + G < cnt ? first + G : cnt) - 1;
  Val<N> carry;
  if (above != nullptr && g + 1 < cnt_above)
    load_val_full<N>(above + (g + 1) * full_val_doubles<N>(), carry);
  else
    zero_val<N>(carry);
  // composite of the maps of this chunk (x_{first} -> x_{last+1})
  double P[N * N], pv[N];
  constexpr int PM = N * N + N;
#pragma unroll
  for (int i = 0; i < N * N; ++i) P[i] = (i % (N + 1) == 0) ? 1.0 : 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) pv[i] = 0.0;
  Elem<N> e;
  Val<N> nv;
  double Psi[N * N], alpha[N];
  for (int64_t k = last; k >= first; --k) {
    src.load(k, e);
    double zinc;
    combine_value<N, GT>(e, carry, nv, Psi, alpha, &zinc);
    store_val_public<N>(o, k, nv);
    if (o.zeta_inc && o.zeta) o.zeta[k] = zinc;
    if (o.maps != nullptr && k < o.T) {
      double* mp = o.maps + k * PM;
#pragma unroll
      for (int i = 0; i < N * N; ++i) mp[i] = Psi[i];
#pragma unroll
      for (int i = 0; i < N; ++i) mp[N * N + i] = alpha[i];
      // (P, pv) <- (P Psi, P alpha + pv)
      double P2[N * N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double s = pv[i];
#pragma unroll
        for (int l = 0; l < N; ++l) s = fma(P[i * N + l], alpha[l], s);
        pv[i] = s;
#pragma unroll
        for (int j = 0; j < N; ++j) {
          double t = 0.0;
#pragma unroll
          for (int l = 0; l < N; ++l) t = fma(P[i * N + l], Psi[l * N + j], t);
          P2[i * N + j] = t;
        }
      }
#pragma unroll
      for (int i = 0; i < N * N; ++i) P[i] = P2[i];
    }
    carry = nv;
  }
  if (o.composite != nullptr && last + 1 <= o.T) {
    // chunk g maps x_{first} to x_{last+1}; only chunks that end at or before T
    double* cp = o.composite + g * PM;
#pragma unroll
    for (int i = 0; i < N * N; ++i) cp[i] = P[i];
#pragma unroll
    for (int i = 0; i < N; ++i) cp[N * N + i] = pv[i];
  }
}

// Upper-level down-sweep, one thread per group: suffix values of the group's
// records (full layout) from the carry of the level above, written in the
// full value layout.
template <int N, typename GT = double>
__global__ void __launch_bounds__(128) down_vals_upper_kernel(SrcFull<N> src, int64_t cnt, int G,
                                                              const double* __restrict__ above, int64_t cnt_above,
                                                              double* __restrict__ vals) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t first = g * G;
  if (first >= cnt) return;
  const int64_t last = (first + G < cnt ? first + G : cnt) - 1;
  Val<N> carry, nv;
  if (above != nullptr && g + 1 < cnt_above)
    load_val_full<N>(above + (g + 1) * full_val_doubles<N>(), carry);
  else
    zero_val<N>(carry);
  Elem<N> e;
  double Psi[N * N], alpha[N];
  for (int64_t k = last; k >= first; --k) {
    src.load(k, e);
    combine_value<N, GT>(e, carry, nv, Psi, alpha);
    store_val_full<N>(vals + k * full_val_doubles<N>(), nv);
    carry = nv;
  }
}

// ---------------------------------------------------------------------------
// affine-map (trajectory) scan kernels
// ---------------------------------------------------------------------------

// comp[g] = map[last] o ... o map[first]  (apply first map first)
template <int N>
__global__ void __launch_bounds__(128) reduce_maps_kernel(const double* __restrict__ maps, int64_t cnt, int G,
                                                          double* __restrict__ comp) {
  constexpr int PM = N * N + N;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t first = g * G;
  if (first >= cnt) return;
  const int64_t last = (first + G < cnt ? first + G : cnt) - 1;
  double P[N * N], p[N];
  const double* m0 = maps + first * PM;
#pragma unroll
  for (int i = 0; i < N * N; ++i) P[i] = m0[i];
#pragma unroll
  for (int i = 0; i < N; ++i) p[i] = m0[N * N + i];
  for (int64_t k = first + 1; k <= last; ++k) {
    const double* mk = maps + k * PM;
    double Ps[N * N], ps[N];
    // x -> Psi_k (P x + p) + alpha_k
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = mk[N * N + i];
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(mk[i * N + l], p[l], s);
      ps[i] = s;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        double t = 0.0;
#pragma unroll
        for (int l = 0; l < N; ++l) t = fma(mk[i * N + l], P[l * N + j], t);
        Ps[i * N + j] = t;
      }
    }
#pragma unroll
    for (int i = 0; i < N * N; ++i) P[i] = Ps[i];
#pragma unroll
    for (int i = 0; i < N; ++i) p[i] = ps[i];
  }
  double* out = comp + g * PM;
#pragma unroll
  for (int i = 0; i < N * N; ++i) out[i] = P[i];
#pragma unroll
  for (int i = 0; i < N; ++i) out[N * N + i] = p[i];
}

// starts[i] for i in group g: starts[first] = above[g] (or x_in at the top),
// starts[i+1] = map_i(starts[i]); the group holding the last map also writes
// starts[cnt].
template <int N>
__global__ void __launch_bounds__(128) down_maps_kernel(const double* __restrict__ maps, int64_t cnt, int G,
                                                        const double* __restrict__ above,
                                                        const double* __restrict__ x_in,
                                                        double* __restrict__ starts) {
  constexpr int PM = N * N + N;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t first = g * G;
  if (first >= cnt) return;
  const int64_t last = (first + G < cnt ? first + G : cnt) - 1;
  double x[N];
  const double* xs = above ? above + g * N : x_in;
#pragma unroll
  for (int i = 0; i < N; ++i) x[i] = xs[i];
  for (int64_t k = first; k <= last; ++k) {
#pragma unroll
    for (int i = 0; i < N; ++i) starts[k * N + i] = x[i];
    const double* mk = maps + k * PM;
    double y[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = mk[N * N + i];
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(mk[i * N + l], x[l], s);
      y[i] = s;
    }
#pragma unroll
    for (int i = 0; i < N; ++i) x[i] = y[i];
  }
  if (last == cnt - 1) {
#pragma unroll
    for (int i = 0; i < N; ++i) starts[cnt * N + i] = x[i];
  }
}

// Optimal-state maps of the sub-intervals of one chunk from given S, v
// (standalone trajectory call), with the chunk composite.
template <int N>
__global__ void __launch_bounds__(128) maps_from_values_kernel(SrcPublic<N> src, int64_t T, int G,
                                                               const double* __restrict__ S,
                                                               const double* __restrict__ v, double* maps,
                                                               double* composite) {
  constexpr int PM = N * N + N;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t first = g * G;
  if (first > T) return;
  const int64_t last = (first + G < T + 1 ? first + G : T + 1) - 1;
  double P[N * N], pv[N];
#pragma unroll
  for (int i = 0; i < N * N; ++i) P[i] = (i % (N + 1) == 0) ? 1.0 : 0.0;
#pragma unroll
  for (int i = 0; i < N; ++i) pv[i] = 0.0;
  Elem<N> e;
  Val<N> V, nv;
  double Psi[N * N], alpha[N];
  for (int64_t k = (last < T ? last : T - 1); k >= first; --k) {
    src.load(k, e);
    const double* Sk = S + (k + 1) * N * N;
#pragma unroll
    for (int i = 0; i < N; ++i)
#pragma unroll
      for (int j = i; j < N; ++j) V.S[sidx<N>(i, j)] = 0.5 * (Sk[i * N + j] + Sk[j * N + i]);
#pragma unroll
    for (int i = 0; i < N; ++i) V.v[i] = v[(k + 1) * N + i];
    V.zeta = 0.0;
    combine_value<N>(e, V, nv, Psi, alpha);
    double* mp = maps + k * PM;
#pragma unroll
    for (int i = 0; i < N * N; ++i) mp[i] = Psi[i];
#pragma unroll
    for (int i = 0; i < N; ++i) mp[N * N + i] = alpha[i];
    double P2[N * N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = pv[i];
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(P[i * N + l], alpha[l], s);
      pv[i] = s;
#pragma unroll
      for (int j = 0; j < N; ++j) {
        double t = 0.0;
#pragma unroll
        for (int l = 0; l < N; ++l) t = fma(P[i * N + l], Psi[l * N + j], t);
        P2[i * N + j] = t;
      }
    }
#pragma unroll
    for (int i = 0; i < N * N; ++i) P[i] = P2[i];
  }
  if (composite != nullptr && last + 1 <= T) {
    double* cp = composite + g * PM;
#pragma unroll
    for (int i = 0; i < N * N; ++i) cp[i] = P[i];
#pragma unroll
    for (int i = 0; i < N; ++i) cp[N * N + i] = pv[i];
  }
}

// Level-0 apply: states of every boundary in chunk g from its start state,
// controls u_k = Ku (v_k - S_k x_k), and (thread 0) the optimal cost.
template <int N>
__global__ void __launch_bounds__(128) final_traj_kernel(const double* __restrict__ maps, int64_t T, int G,
                                                         const double* __restrict__ starts1,
                                                         const double* __restrict__ x0,
                                                         const double* __restrict__ S,
                                                         const double* __restrict__ v,
                                                         const double* __restrict__ zeta, const double* __restrict__ Ku,
                                                         int32_t Ku_per_boundary, int32_t m, double* __restrict__ x,
                                                         double* __restrict__ u, double* __restrict__ cost) {
  constexpr int PM = N * N + N;
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t first = g * G;
  if (first > T) return;
  const int64_t last = (first + G < T + 1 ? first + G : T + 1) - 1;
  double xc[N];
  const double* xs = starts1 ? starts1 + g * N : x0;
#pragma unroll
  for (int i = 0; i < N; ++i) xc[i] = xs[i];
  bool ok = true;
  for (int64_t k = first; k <= last; ++k) {
#pragma unroll
    for (int i = 0; i < N; ++i) {
      x[k * N + i] = xc[i];
      ok = ok && isfinite(xc[i]);
    }
    if (u != nullptr) {
      double e[N];
      const double* Sk = S + k * N * N;
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double s = v[k * N + i];
#pragma unroll
        for (int l = 0; l < N; ++l) s = fma(-Sk[i * N + l], xc[l], s);
        e[i] = s;
      }
      const double* Kk = Ku + (Ku_per_boundary ? k * m * N : 0);
      for (int a = 0; a < m; ++a) {
        double s = 0.0;
#pragma unroll
        for (int l = 0; l < N; ++l) s = fma(Kk[a * N + l], e[l], s);
        u[k * m + a] = s;
      }
    }
    if (k < T) {
      const double* mk = maps + k * PM;
      double y[N];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        double s = mk[N * N + i];
#pragma unroll
        for (int l = 0; l < N; ++l) s = fma(mk[i * N + l], xc[l], s);
        y[i] = s;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) xc[i] = y[i];
    }
  }
  if (!ok) flag(kStatusNonFinite);
  if (g == 0 && cost != nullptr) {
    // V(x0, t0) = zeta_0 + 1/2 x0'S_0 x0 - v_0'x0
    double c = zeta ? zeta[0] : 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(S[i * N + l], x0[l], s);
      c = fma(x0[i], fma(0.5, s, -v[i]), c);
    }
    *cost = c;
  }
}

// ---------------------------------------------------------------------------
// host drivers
// ---------------------------------------------------------------------------

static unsigned blocks_for(int64_t threads) { return (unsigned)ceil_div(threads, 128); }

// Workspace plan of the scans (byte offsets from the scan region start).
struct ScanPlan {
  int G0;
  int64_t T;
  // value levels >= 1
  int nlev;
  int64_t cnt[64];
  size_t off_agg[64], off_val[64];
  // trajectory
  size_t off_maps;  // level-0 maps [T]
  int tlev;
  int64_t tcnt[64];                 // number of maps at trajectory level l (l >= 1)
  size_t off_tmap[64], off_tstart[64];
  size_t bytes;
};

template <int N>
static ScanPlan make_plan(int64_t T, bool with_traj) {
  ScanPlan pl;
  pl.G0 = level0_group(T);
  pl.T = T;
  size_t off = 0;
  const size_t PE = sizeof(double) * full_elem_doubles<N>();
  const size_t PV = sizeof(double) * full_val_doubles<N>();
  const size_t PM = sizeof(double) * (N * N + N);
  int64_t c = T + 1;
  int G = pl.G0;
  pl.nlev = 0;
  while (c > G) {
    const int64_t nc = ceil_div(c, G);
    pl.cnt[pl.nlev] = nc;
    pl.off_agg[pl.nlev] = off;
    off = align_up(off + nc * PE);
    pl.off_val[pl.nlev] = off;
    off = align_up(off + nc * PV);
    ++pl.nlev;
    c = nc;
    G = kUpperGroup;
  }
  pl.off_maps = off;
  pl.tlev = 0;
  if (with_traj) {
    off = align_up(off + (size_t)T * PM);
    // level-1 maps: chunk composites, one per level-0 chunk that ends <= T
    int64_t mc = ceil_div(T + 1, pl.G0) - 1;
    while (mc > 0) {
      pl.tcnt[pl.tlev] = mc;
      pl.off_tmap[pl.tlev] = off;
      off = align_up(off + mc * PM);
      pl.off_tstart[pl.tlev] = off;
      off = align_up(off + (mc + 1) * sizeof(double) * N);
      ++pl.tlev;
      if (mc <= kUpperGroup) break;
      mc = ceil_div(mc, kUpperGroup);
    }
  }
  pl.bytes = align_up(off);
  return pl;
}

// Upper levels with fewer pairs than this run one warp per combination (the
// level is then latency-bound: a warp spreads one combination's products
// over its lanes, shortening the dependent FP64 chain); larger levels run one
// thread per pair (throughput-bound: a thread-per-pair warp instruction
// serves 32 combinations).  Both read and write the same full-matrix records.
// A thread's chain grows as n^3 (~5 k FP64 instructions at n = 8, ~155 us at
// 64 cycles each, against ~0.6 k at n = 4), so the crossing moves up with n.
// For n <= 3 a thread's combination is already short, and the warp version
// is not faster at any level size.
template <int N>
constexpr int64_t team_level_below() {
  return N >= 8 ? 8192 : (N >= 4 ? 2048 : 0);
}

// Level 0 (chunks of G0 elements, one thread each, register-resident) and the
// pairwise upper levels.
template <int N, typename GT = double>
static void value_scan(const ScanPlan& pl, const ElemPtrs& el, const DownOut& out0, char* ws, cudaStream_t st) {
  const int64_t T = pl.T;
  SrcPublic<N> s0{el};
  // reduce up the levels
  int64_t c = T + 1;
  for (int l = 0; l < pl.nlev; ++l) {
    double* agg = (double*)(ws + pl.off_agg[l]);
    if (l == 0) {
      reduce_elems_kernel<N, SrcPublic<N>, GT><<<blocks_for(pl.cnt[0]), 128, 0, st>>>(s0, c, pl.G0, agg);
      count_launch();
    } else if (pl.cnt[l] < team_level_below<N>()) {
      team_upper_reduce<N, GT>((const double*)(ws + pl.off_agg[l - 1]), c, agg, st);
    } else {
      SrcFull<N> sf{(const double*)(ws + pl.off_agg[l - 1])};
      reduce_elems_kernel<N, SrcFull<N>, GT><<<blocks_for(pl.cnt[l]), 128, 0, st>>>(sf, c, kUpperGroup, agg);
      count_launch();
    }
    c = pl.cnt[l];
  }
  // down the levels: top level first (one group, zero carry)
  for (int l = pl.nlev; l >= 1; --l) {
    const double* above = (l < pl.nlev) ? (const double*)(ws + pl.off_val[l]) : nullptr;
    const int64_t cabove = (l < pl.nlev) ? pl.cnt[l] : 0;
    const int64_t cl = pl.cnt[l - 1];
    const int64_t groups = ceil_div(cl, kUpperGroup);
    double* vals = (double*)(ws + pl.off_val[l - 1]);
    if (groups < team_level_below<N>()) {
      team_upper_down<N, GT>((const double*)(ws + pl.off_agg[l - 1]), cl, above, cabove, vals, st);
    } else {
      SrcFull<N> sf{(const double*)(ws + pl.off_agg[l - 1])};
      down_vals_upper_kernel<N, GT><<<blocks_for(groups), 128, 0, st>>>(sf, cl, kUpperGroup, above, cabove, vals);
      count_launch();
    }
  }
  const double* above = pl.nlev > 0 ? (const double*)(ws + pl.off_val[0]) : nullptr;
  const int64_t cabove = pl.nlev > 0 ? pl.cnt[0] : 0;
  down_values_kernel<N, SrcPublic<N>, GT><<<blocks_for(ceil_div(T + 1, pl.G0)), 128, 0, st>>>(
      s0, T + 1, pl.G0, above, cabove, out0);
  count_launch();
}

template <int N>
static void traj_scan(const ScanPlan& pl, const double* x0, const double* S, const double* v, const double* zeta,
                      const Coefs& cf, int32_t m, double* x, double* u, double* cost, char* ws, cudaStream_t st) {
  const int64_t T = pl.T;
  const double* maps0 = (const double*)(ws + pl.off_maps);
  // reduce the chunk composites up the trajectory levels (thread or warp per
  // composition by level size, as for the value levels)
  for (int l = 1; l < pl.tlev; ++l) {
    if (pl.tcnt[l] < team_level_below<N>()) {
      team_maps_reduce<N>((const double*)(ws + pl.off_tmap[l - 1]), pl.tcnt[l - 1], kUpperGroup,
                          (double*)(ws + pl.off_tmap[l]), st);
    } else {
      reduce_maps_kernel<N><<<blocks_for(pl.tcnt[l]), 128, 0, st>>>((const double*)(ws + pl.off_tmap[l - 1]),
                                                                      pl.tcnt[l - 1], kUpperGroup,
                                                                      (double*)(ws + pl.off_tmap[l]));
      count_launch();
    }
  }
  // starts down the levels
  for (int l = pl.tlev - 1; l >= 0; --l) {
    const double* above = (l + 1 < pl.tlev) ? (const double*)(ws + pl.off_tstart[l + 1]) : nullptr;
    const int G = (l + 1 < pl.tlev) ? kUpperGroup : (int)pl.tcnt[l];
    const int64_t groups = ceil_div(pl.tcnt[l], G);
    if (groups < team_level_below<N>()) {
      team_maps_down<N>((const double*)(ws + pl.off_tmap[l]), pl.tcnt[l], G, above, x0,
                        (double*)(ws + pl.off_tstart[l]), st);
    } else {
      down_maps_kernel<N><<<blocks_for(groups), 128, 0, st>>>((const double*)(ws + pl.off_tmap[l]), pl.tcnt[l], G,
                                                             above, x0, (double*)(ws + pl.off_tstart[l]));
      count_launch();
    }
  }
  const double* starts1 = pl.tlev > 0 ? (const double*)(ws + pl.off_tstart[0]) : nullptr;
  final_traj_kernel<N><<<blocks_for(ceil_div(T + 1, pl.G0)), 128, 0, st>>>(
      maps0, T, pl.G0, starts1, x0, S, v, zeta, cf.Ku, cf.Ku_per_boundary, m, x, u, cost);
  count_launch();
}

static thread_local bool t_mixed = false;
void set_mixed_precision(bool on) { t_mixed = on; }
bool mixed_precision() { return t_mixed; }

template <int N>
static cudaError_t run_n(const lqt_problem& p, const Coefs& cf, const ElemPtrs& el, double* S, double* v,
                         double* zeta, const double* x0, double* x, double* u, double* cost, bool do_value,
                         bool do_traj, char* ws, cudaStream_t st) {
  const ScanPlan pl = make_plan<N>(p.T, do_traj);
  double* maps0 = (double*)(ws + pl.off_maps);
  double* comp1 = pl.tlev > 0 ? (double*)(ws + pl.off_tmap[0]) : nullptr;
  if (do_value) {
    DownOut o{};
    o.S = S; o.v = v; o.zeta = zeta; o.T = p.T;
    o.maps = do_traj ? maps0 : nullptr;
    o.composite = do_traj ? comp1 : nullptr;
    if (t_mixed)
      value_scan<N, float>(pl, el, o, ws, st);
    else
      value_scan<N, double>(pl, el, o, ws, st);
  } else if (do_traj) {
    SrcPublic<N> s0{el};
    maps_from_values_kernel<N><<<blocks_for(ceil_div(p.T + 1, pl.G0)), 128, 0, st>>>(s0, p.T, pl.G0, S, v, maps0,
                                                                                     comp1);
    count_launch();
  }
  if (do_traj) traj_scan<N>(pl, x0, S, v, zeta, cf, p.m, x, u, cost, ws, st);
  return cudaGetLastError();
}

// Generic forward affine-map scan: states[0] = x_in, states[k+1] = map_k(states[k])
// for k < cnt (maps [cnt][N*N+N]), as pairwise reduce levels + down-sweeps.
template <int N>
static void affine_scan_n(const double* maps, int64_t cnt, const double* x_in, double* states, char* ws,
                          size_t& off, cudaStream_t st) {
  constexpr int PM = N * N + N;
  const int G = kUpperGroup;
  int nlev = 0;
  int64_t c[64];
  double* lv[64];
  double* sv[64];
  int64_t mc = cnt;
  const double* prev = maps;
  while (mc > G) {
    const int64_t nc = ceil_div(mc, G);
    double* out = (double*)(ws + off);
    off = align_up(off + nc * PM * sizeof(double));
    if (nc < team_level_below<N>()) {
      team_maps_reduce<N>(prev, mc, G, out, st);
    } else {
      reduce_maps_kernel<N><<<blocks_for(nc), 128, 0, st>>>(prev, mc, G, out);
      count_launch();
    }
    c[nlev] = nc;
    lv[nlev] = out;
    sv[nlev] = (double*)(ws + off);
    off = align_up(off + (nc + 1) * N * sizeof(double));
    prev = out;
    mc = nc;
    ++nlev;
  }
  {
    const double* tm = nlev ? lv[nlev - 1] : maps;
    const int64_t tc = nlev ? c[nlev - 1] : cnt;
    double* ts = nlev ? sv[nlev - 1] : states;
    down_maps_kernel<N><<<1, 128, 0, st>>>(tm, tc, (int)tc, nullptr, x_in, ts);
    count_launch();
  }
  for (int l = nlev - 1; l >= 0; --l) {
    const double* mp = (l == 0) ? maps : lv[l - 1];
    const int64_t mcnt = (l == 0) ? cnt : c[l - 1];
    double* outst = (l == 0) ? states : sv[l - 1];
    if (ceil_div(mcnt, G) < team_level_below<N>()) {
      team_maps_down<N>(mp, mcnt, G, sv[l], x_in, outst, st);
    } else {
      down_maps_kernel<N><<<blocks_for(ceil_div(mcnt, G)), 128, 0, st>>>(mp, mcnt, G, sv[l], x_in, outst);
      count_launch();
    }
  }
}

// Problem b's boundary map (index off[b+1] - 1 of the concatenation, its
// terminal element) becomes x -> x0 of problem b+1.
__global__ void boundary_patch_kernel(int n, double* maps, BoundaryPatch pt) {
  const int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (b + 1 >= pt.B) return;
  const int64_t k = pt.off[b + 1] - 1;
  double* mp = maps + k * (n * n + n);
  for (int i = 0; i < n * n; ++i) mp[i] = 0.0;
  const double* x0 = pt.probs[b + 1].x0;
  for (int i = 0; i < n; ++i) mp[n * n + i] = x0[i];
}

void launch_boundary_patch(int n, double* maps, const BoundaryPatch& patch, cudaStream_t st) {
  if (patch.B < 2) return;
  boundary_patch_kernel<<<(unsigned)ceil_div(patch.B, 128), 128, 0, st>>>(n, maps, patch);
  count_launch();
}

template <int N>
static cudaError_t concat_n(int64_t Tcat, const ElemPtrs& el, double* S, double* v, double* zeta,
                            const double* x0_first, double* x, const BoundaryPatch& patch, char* ws,
                            cudaStream_t st) {
  const ScanPlan pl = make_plan<N>(Tcat, true);
  double* maps0 = (double*)(ws + pl.off_maps);
  DownOut o{};
  o.S = S; o.v = v; o.zeta = zeta; o.T = Tcat; o.maps = maps0; o.composite = nullptr; o.zeta_inc = 1;
  value_scan<N>(pl, el, o, ws, st);
  launch_boundary_patch(N, maps0, patch, st);
  if (pl.tlev > 0) {
    const int64_t cnt = pl.tcnt[0] * pl.G0 < Tcat ? pl.tcnt[0] * pl.G0 : Tcat;
    reduce_maps_kernel<N><<<blocks_for(pl.tcnt[0]), 128, 0, st>>>(maps0, cnt, pl.G0, (double*)(ws + pl.off_tmap[0]));
    count_launch();
  }
  Coefs cf{};
  traj_scan<N>(pl, x0_first, S, v, zeta, cf, 0, x, nullptr, nullptr, ws, st);
  return cudaGetLastError();
}

size_t concat_workspace_bytes(int32_t n, int64_t Tcat) {
  if (n == 16 || n == 64) return team_concat_workspace_bytes(n, Tcat);
  return scan_workspace_bytes(n, Tcat, true);
}

cudaError_t concat_scan(int32_t n, int64_t Tcat, const ElemPtrs& el, double* S, double* v, double* zeta,
                        const double* x0_first, double* x, const BoundaryPatch& patch, char* ws, cudaStream_t st) {
  switch (n) {
    case 1: return concat_n<1>(Tcat, el, S, v, zeta, x0_first, x, patch, ws, st);
    case 2: return concat_n<2>(Tcat, el, S, v, zeta, x0_first, x, patch, ws, st);
    case 3: return concat_n<3>(Tcat, el, S, v, zeta, x0_first, x, patch, ws, st);
    case 4: return concat_n<4>(Tcat, el, S, v, zeta, x0_first, x, patch, ws, st);
    case 8: return concat_n<8>(Tcat, el, S, v, zeta, x0_first, x, patch, ws, st);
    case 16:
    case 64: return team_concat_scan(n, Tcat, el, S, v, zeta, x0_first, x, patch, ws, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t affine_scan_bytes(int n, int64_t cnt) {
  const size_t PM = (size_t)(n * n + n) * sizeof(double);
  size_t off = 0;
  int64_t mc = cnt;
  while (mc > kUpperGroup) {
    const int64_t nc = ceil_div(mc, kUpperGroup);
    off = align_up(off + nc * PM);
    off = align_up(off + (nc + 1) * n * sizeof(double));
    mc = nc;
  }
  return off + 256;
}

cudaError_t affine_scan_states(int n, const double* maps, int64_t cnt, const double* x_in, double* states, char* ws,
                               size_t& off, cudaStream_t st) {
  switch (n) {
    case 1: affine_scan_n<1>(maps, cnt, x_in, states, ws, off, st); break;
    case 2: affine_scan_n<2>(maps, cnt, x_in, states, ws, off, st); break;
    case 3: affine_scan_n<3>(maps, cnt, x_in, states, ws, off, st); break;
    case 4: affine_scan_n<4>(maps, cnt, x_in, states, ws, off, st); break;
    case 8: affine_scan_n<8>(maps, cnt, x_in, states, ws, off, st); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_maps_from_values(const lqt_problem& p, const ElemPtrs& el, const double* S, const double* v,
                                    double* maps, cudaStream_t st) {
  const int G = 2;
  const int64_t groups = ceil_div(p.T + 1, G);
  switch (p.n) {
#define LQT_MFV(NN)                                                                                       \
  case NN:                                                                                                \
    maps_from_values_kernel<NN><<<blocks_for(groups), 128, 0, st>>>(SrcPublic<NN>{el}, p.T, G, S, v, maps, \
                                                                    nullptr);                            \
    break;
    LQT_MFV(1)
    LQT_MFV(2)
    LQT_MFV(3)
    LQT_MFV(4)
    LQT_MFV(8)
#undef LQT_MFV
    default: return cudaErrorInvalidValue;
  }
  count_launch();
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Method 2 (Sec. IV-E, eq. Opt_trajectory_method2): prefix scan of the
// forward-ODE elements and the optimal states from the prefixes
// ---------------------------------------------------------------------------

// Levels of the prefix scan over T elements: chunk aggregates at level 0,
// pairs above; per level the aggregates and their exclusive prefixes (full
// records).
struct PrefixPlan {
  int G0;
  int64_t T;
  int nlev;
  int64_t cnt[64];
  size_t off_agg[64], off_pre[64];
  size_t bytes;
};

template <int N>
static PrefixPlan make_prefix_plan(int64_t T) {
  PrefixPlan pl{};
  pl.G0 = level0_group(T);
  pl.T = T;
  const size_t PE = sizeof(double) * full_elem_doubles<N>();
  size_t off = 0;
  int64_t c = T;
  int G = pl.G0;
  while (c > G) {
    const int64_t nc = ceil_div(c, G);
    pl.cnt[pl.nlev] = nc;
    pl.off_agg[pl.nlev] = off;
    off = align_up(off + nc * PE);
    pl.off_pre[pl.nlev] = off;
    off = align_up(off + nc * PE);
    ++pl.nlev;
    c = nc;
    G = kUpperGroup;
  }
  pl.bytes = align_up(off);
  return pl;
}

// Exclusive prefixes of the level-l aggregates, one thread per pair (the
// large levels; the small ones run one warp per pair in lqt_team.cu):
// pre[2g] = pre_up[g], pre[2g+1] = pre_up[g] (x) agg[2g].
template <int N>
__global__ void __launch_bounds__(128) prefix_down_kernel(const double* __restrict__ agg, int64_t cnt,
                                                          const double* __restrict__ pre_up,
                                                          double* __restrict__ pre) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (2 * g >= cnt) return;
  constexpr int FE = full_elem_doubles<N>();
  Elem<N> left, e;
  if (pre_up) {
    load_full<N>(pre_up + g * FE, left);
  } else {
#pragma unroll
    for (int i = 0; i < N * N; ++i) left.A[i] = (i % (N + 1) == 0) ? 1.0 : 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      left.b[i] = 0.0;
      left.eta[i] = 0.0;
    }
#pragma unroll
    for (int i = 0; i < Dim<N>::NS; ++i) {
      left.C[i] = 0.0;
      left.J[i] = 0.0;
    }
    left.zeta = 0.0;
  }
  store_full<N>(pre + 2 * g * FE, left);
  if (2 * g + 1 < cnt) {
    load_full<N>(agg + 2 * g * FE, e);
    combine<N>(left, e, e);
    store_full<N>(pre + (2 * g + 1) * FE, e);
  }
}

struct Method2Args {
  ElemPtrs el;  // forward-ODE elements, T of them
  int64_t T;
  int G;
  const double* pre0;  // exclusive prefixes of the level-0 chunks (full records), or null (one chunk)
  const double *S, *v, *zeta, *x0;
  const double* Ku;
  int32_t Ku_per_boundary, m;
  double *x, *u, *cost;
};

// x_k = (I + C S_k)^-1 (A x0 + b + C v_k) for the prefix (A, b, C) = V(., t_0;
// ., t_k), then u_k = U^-1 L^T (v_k - S_k x_k).  Returns false if x_k is not finite.
template <int N>
__device__ __forceinline__ bool method2_state(const Method2Args& a, int64_t k, const Prefix<N>& P) {
  const double* Sk = a.S + k * N * N;
  const double* vk = a.v + k * N;
  double W[N * N], r[N];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    double s = P.b[i];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      s = fma(P.A[i * N + l], a.x0[l], s);
      s = fma(P.C[sidx<N>(i, l)], vk[l], s);
    }
    r[i] = s;
#pragma unroll
    for (int j = 0; j < N; ++j) {
      double w = (i == j) ? 1.0 : 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) w = fma(P.C[sidx<N>(i, l)], Sk[l * N + j], w);
      W[i * N + j] = w;
    }
  }
  lu_solve<N, 1>(W, r);
  bool ok = true;
#pragma unroll
  for (int i = 0; i < N; ++i) {
    a.x[k * N + i] = r[i];
    ok = ok && isfinite(r[i]);
  }
  if (a.u) {
    double e[N];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = vk[i];
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(-Sk[i * N + l], r[l], s);
      e[i] = s;
    }
    const double* Kk = a.Ku + (a.Ku_per_boundary ? k * a.m * N : 0);
    for (int q = 0; q < a.m; ++q) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(Kk[q * N + l], e[l], s);
      a.u[k * a.m + q] = s;
    }
  }
  return ok;
}

// One thread per level-0 chunk: fold the chunk's elements left to right onto
// the prefix before the chunk, emitting the state at every boundary.
template <int N>
__global__ void __launch_bounds__(128) method2_kernel(Method2Args a) {
  const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t first = g * a.G;
  if (first >= a.T) return;
  const int64_t last = (first + a.G < a.T ? first + a.G : a.T) - 1;
  Prefix<N> P;
  if (a.pre0)
    load_prefix_full<N>(a.pre0 + g * full_elem_doubles<N>(), P);
  else
    identity_prefix<N>(P);
  SrcPublic<N> src{a.el};
  Elem<N> e;
  bool ok = true;
  for (int64_t k = first; k <= last; ++k) {
    ok = method2_state<N>(a, k, P) && ok;
    src.load(k, e);
    combine_prefix<N>(P, e);
  }
  if (last == a.T - 1) ok = method2_state<N>(a, a.T, P) && ok;
  if (!ok) flag(kStatusNonFinite);
  if (g == 0 && a.cost != nullptr) {
    double c = a.zeta ? a.zeta[0] : 0.0;
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double s = 0.0;
#pragma unroll
      for (int l = 0; l < N; ++l) s = fma(a.S[i * N + l], a.x0[l], s);
      c = fma(a.x0[i], fma(0.5, s, -a.v[i]), c);
    }
    *a.cost = c;
  }
}

template <int N>
static cudaError_t method2_n(const lqt_problem& p, const Coefs& cf, const ElemPtrs& fwd, const double* S,
                             const double* v, const double* zeta, const double* x0, double* x, double* u,
                             double* cost, char* ws, cudaStream_t st) {
  const PrefixPlan pl = make_prefix_plan<N>(p.T);
  SrcPublic<N> s0{fwd};
  int64_t c = p.T;
  for (int l = 0; l < pl.nlev; ++l) {
    double* agg = (double*)(ws + pl.off_agg[l]);
    if (l == 0) {
      reduce_elems_kernel<N, SrcPublic<N>, double><<<blocks_for(pl.cnt[0]), 128, 0, st>>>(s0, c, pl.G0, agg);
      count_launch();
    } else if (pl.cnt[l] < team_level_below<N>()) {
      team_upper_reduce<N, double>((const double*)(ws + pl.off_agg[l - 1]), c, agg, st);
    } else {
      SrcFull<N> sf{(const double*)(ws + pl.off_agg[l - 1])};
      reduce_elems_kernel<N, SrcFull<N>, double><<<blocks_for(pl.cnt[l]), 128, 0, st>>>(sf, c, kUpperGroup, agg);
      count_launch();
    }
    c = pl.cnt[l];
  }
  for (int l = pl.nlev - 1; l >= 0; --l) {
    const double* up = l + 1 < pl.nlev ? (const double*)(ws + pl.off_pre[l + 1]) : nullptr;
    const int64_t pairs = ceil_div(pl.cnt[l], 2);
    if (pairs < team_level_below<N>()) {
      team_prefix_down<N>((const double*)(ws + pl.off_agg[l]), pl.cnt[l], up, (double*)(ws + pl.off_pre[l]), st);
    } else {
      prefix_down_kernel<N><<<blocks_for(pairs), 128, 0, st>>>((const double*)(ws + pl.off_agg[l]), pl.cnt[l], up,
                                                               (double*)(ws + pl.off_pre[l]));
      count_launch();
    }
  }
  Method2Args a{};
  a.el = fwd; a.T = p.T; a.G = pl.G0;
  a.pre0 = pl.nlev > 0 ? (const double*)(ws + pl.off_pre[0]) : nullptr;
  a.S = S; a.v = v; a.zeta = zeta; a.x0 = x0;
  a.Ku = cf.Ku; a.Ku_per_boundary = cf.Ku_per_boundary; a.m = p.m;
  a.x = x; a.u = u; a.cost = cost;
  method2_kernel<N><<<blocks_for(ceil_div(p.T, pl.G0)), 128, 0, st>>>(a);
  count_launch();
  return cudaGetLastError();
}

size_t prefix_workspace_bytes(int n, int64_t T) {
  switch (n) {
    case 1: return make_prefix_plan<1>(T).bytes;
    case 2: return make_prefix_plan<2>(T).bytes;
    case 3: return make_prefix_plan<3>(T).bytes;
    case 4: return make_prefix_plan<4>(T).bytes;
    case 8: return make_prefix_plan<8>(T).bytes;
    case 16:
    case 64: return team_prefix_workspace_bytes(n, T);
    default: return 0;
  }
}

cudaError_t run_method2(const lqt_problem& p, const Coefs& cf, const ElemPtrs& fwd, const double* S,
                        const double* v, const double* zeta, const double* x0, double* x, double* u, double* cost,
                        char* ws, cudaStream_t st) {
  switch (p.n) {
    case 1: return method2_n<1>(p, cf, fwd, S, v, zeta, x0, x, u, cost, ws, st);
    case 2: return method2_n<2>(p, cf, fwd, S, v, zeta, x0, x, u, cost, ws, st);
    case 3: return method2_n<3>(p, cf, fwd, S, v, zeta, x0, x, u, cost, ws, st);
    case 4: return method2_n<4>(p, cf, fwd, S, v, zeta, x0, x, u, cost, ws, st);
    case 8: return method2_n<8>(p, cf, fwd, S, v, zeta, x0, x, u, cost, ws, st);
    case 16:
    case 64: return team_run_method2(p, cf, fwd, S, v, zeta, x0, x, u, cost, ws, st);
    default: return cudaErrorInvalidValue;
  }
}

size_t scan_workspace_bytes(int32_t n, int64_t T, bool with_traj) {
  switch (n) {
    case 1: return make_plan<1>(T, with_traj).bytes;
    case 2: return make_plan<2>(T, with_traj).bytes;
    case 3: return make_plan<3>(T, with_traj).bytes;
    case 4: return make_plan<4>(T, with_traj).bytes;
    case 8: return make_plan<8>(T, with_traj).bytes;
    case 16:
    case 64: return team_scan_workspace_bytes(n, T, with_traj);
    default: return 0;
  }
}

cudaError_t run_value_and_traj(const lqt_problem& p, const Layout& lay, const Coefs& cf, const ElemPtrs& el,
                               double* S, double* v, double* zeta, const double* x0, double* x, double* u,
                               double* cost, bool do_value, bool do_traj, const double* S_in, const double* v_in,
                               char* ws, size_t ws_bytes, cudaStream_t st) {
  (void)lay;
  (void)ws_bytes;
  double* Sx = do_value ? S : const_cast<double*>(S_in);
  double* vx = do_value ? v : const_cast<double*>(v_in);
  switch (p.n) {
    case 1: return run_n<1>(p, cf, el, Sx, vx, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
    case 2: return run_n<2>(p, cf, el, Sx, vx, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
    case 3: return run_n<3>(p, cf, el, Sx, vx, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
    case 4: return run_n<4>(p, cf, el, Sx, vx, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
    case 8: return run_n<8>(p, cf, el, Sx, vx, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
    case 16:
    case 64:
      if (!do_value) return cudaErrorNotSupported;
      return team_run_value_and_traj(p, cf, el, Sx, vx, zeta, x0, x, u, cost, do_value, do_traj, ws, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace lqt
