// The batched (multi-right-hand-side) block-Jacobi sweep of Alg. BJ on the FP32 CUDA
// cores.  Per cell the sweep reads six FP32 10x10 blocks, an inverse and three
// [Np x R] slabs, and does (S Np^2 R) FMAs: 3.5 FMAs per byte at Np = 10, R = 32, below the
// FP32 FMA rate per byte of HBM bandwidth, so the sweep is bound by HBM on the CUDA cores
// and gains nothing from tensor-core products.
#include "kcmg_internal.h"

#include <algorithm>
#include <type_traits>

namespace kcmg {

namespace {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
template <typename TI> __device__ __forceinline__ float to_f(TI v);
template <> __device__ __forceinline__ float to_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// ---- cp.async (16/8/4-byte global -> shared copies), per-warp double buffers
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Shape of the CUDA-core sweep: each lane takes CPL consecutive right-hand sides, so
// 32 / CPL lanes own a cell and a warp takes CPL cells (CPL = 4 for 32 columns, 2 for
// other column counts, 1 at Np = 20).  Per cell, shared memory holds the NF off-diagonal
// FP32 blocks (AB bytes) and the stored inverse (DB bytes, TI), each padded to 16 bytes;
// a warp has two stages.
template <int NP, int S, typename TI, int CPL> struct SimtShape {
  static constexpr int NF = S - 1;
  static constexpr int CPW = CPL;                                  // cells per warp
  static constexpr int LPC = 32 / CPL;                             // lanes per cell
  static constexpr int ASZ = NF * NP * NP * 4;
  static constexpr int DSZ = NP * NP * (int)sizeof(TI);
  static constexpr int AB = (ASZ + 15) / 16 * 16;
  static constexpr int DB = (DSZ + 15) / 16 * 16;
  static constexpr int CS = AB + DB;                               // bytes per cell
  static constexpr int WB = 2 * CPW * CS;                          // bytes per warp
  // copy granules: each divides its piece's size and every source offset (the blocks of
  // cell K start at (K S + 1) NP^2 floats, the inverse at K NP^2 entries)
  static constexpr int AG = (NP * NP * 4) % 16 == 0 ? 16 : (NP * NP * 4) % 8 == 0 ? 8 : 4;
  static constexpr int DG = DSZ % 16 == 0 ? 16 : DSZ % 8 == 0 ? 8 : DSZ % 4 == 0 ? 4 : 0;
};

template <int G> __device__ __forceinline__ void cp_async_g(void* dst, const void* src) {
  if (G == 16) cp_async16(dst, src);
  else if (G == 8) cp_async8(dst, src);
  else cp_async4(dst, src);
}

// CPL consecutive columns c0.. of one row: with VEC (R a multiple of CPL, so the offset is
// too) one CPL*4-byte access, else one column at a time; columns >= R read as zero and
// are not written.
template <int CPL, bool VEC> struct Cols {
  static __device__ __forceinline__ void ld(const float* p, int c0, int R, float* v) {
    if (VEC && CPL > 1) {
      if (c0 < R) {
        if (CPL == 4) {
          const float4 t = __ldg(reinterpret_cast<const float4*>(p + c0));
          v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
        } else {
          const float2 t = __ldg(reinterpret_cast<const float2*>(p + c0));
          v[0] = t.x; v[1] = t.y;
        }
      } else {
#pragma unroll
        for (int c = 0; c < CPL; ++c) v[c] = 0.f;
      }
    } else {
#pragma unroll
      for (int c = 0; c < CPL; ++c) v[c] = c0 + c < R ? __ldg(p + c0 + c) : 0.f;
    }
  }
  static __device__ __forceinline__ void st(float* p, int c0, int R, const float* v) {
    if (VEC && CPL > 1) {
      if (c0 >= R) return;
      if (CPL == 4) *reinterpret_cast<float4*>(p + c0) = make_float4(v[0], v[1], v[2], v[3]);
      else *reinterpret_cast<float2*>(p + c0) = make_float2(v[0], v[1]);
    } else {
#pragma unroll
      for (int c = 0; c < CPL; ++c)
        if (c0 + c < R) p[c0 + c] = v[c];
    }
  }
  static __device__ __forceinline__ void st(double* p, int c0, int R, const float* v) {
    if (VEC && CPL > 1) {
      if (c0 >= R) return;
#pragma unroll
      for (int c = 0; c < CPL; c += 2) *reinterpret_cast<double2*>(p + c0 + c) = make_double2(v[c], v[c + 1]);
    } else {
#pragma unroll
      for (int c = 0; c < CPL; ++c)
        if (c0 + c < R) p[c0 + c] = v[c];
    }
  }
};

// two consecutive stored-inverse entries (NP even: 8-byte FP32 / 4-byte BF16 aligned)
template <typename TI> __device__ __forceinline__ float2 ld_pair(const TI* p);
template <> __device__ __forceinline__ float2 ld_pair<float>(const float* p) {
  return *reinterpret_cast<const float2*>(p);
}
template <> __device__ __forceinline__ float2 ld_pair<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(p));
}

// One damped block-Jacobi sweep (Alg. BJ) for R right-hand sides on the FP32 CUDA cores:
//   T = r_K - sum_s A_{K,s} zo_{nbr(K,s)},   zn_K = (1 - om) zo_K + om D_K^{-1} T
// (first sweep: zn_K = om D_K^{-1} r_K).  Each lane keeps its CPL columns of T for all NP
// rows in registers.  The block rows come from shared memory as broadcasts (one 8- or
// 16-byte read per 2-4 FMAs per column), the neighbour slabs, r and zo_K from L2 or HBM
// with one read per row, each in flight during the phase before its use.  Every warp
// walks its own sequence of cell groups with two cp.async stages: the blocks and inverse
// of its next group are in flight while it computes the current one, and the next group's
// neighbour indices are read one group ahead.
// Ac: [C][S][NP][NP] FP32 (cell-major, slot 0 unused here), D: [C][NP][NP] (TI);
// r32, zo: [C*NP][R] FP32; zn: [C*NP][R] (TOUT).  RC > 0: R == RC at compile time.
template <int NP, int S, typename TI, typename TOUT, int CPL, int RC, bool VEC>
__global__ void __launch_bounds__(256) k_msweep_simt(const float* __restrict__ Ac, const TI* __restrict__ D,
                                                     const int* __restrict__ nbr, int C, int Rrt,
                                                     const float* __restrict__ r32, const float* __restrict__ zo,
                                                     TOUT* __restrict__ zn, float om, int first) {
  using Sh = SimtShape<NP, S, TI, CPL>;
  using Cl = Cols<CPL, VEC>;
  constexpr int NF = Sh::NF, CPW = Sh::CPW, LPC = Sh::LPC;
  constexpr bool EVEN = NP % 2 == 0;
  const int R = RC > 0 ? RC : Rrt;
  extern __shared__ __align__(16) unsigned char smem_simt[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int wpb = blockDim.x >> 5;
  unsigned char* wbase = smem_simt + (size_t)warp * Sh::WB;
  const int nunits = (C + CPW - 1) / CPW;
  const int nw = gridDim.x * wpb;
  int u = blockIdx.x * wpb + warp;
  if (u >= nunits) return;
  const int hl = lane / LPC, h = lane - hl * LPC;   // cell of the group, lane within it
  const int c0 = h * CPL;                           // first column of this lane

  // the copies of group un into stage st (all lanes; cells past C are skipped)
  auto load_unit = [&](int un, int st) {
    unsigned char* dst = wbase + (size_t)st * CPW * Sh::CS;
#pragma unroll
    for (int c = 0; c < CPW; ++c) {
      const int K = un * CPW + c;
      if (K >= C) break;
      unsigned char* cd = dst + c * Sh::CS;
      if (!first) {
        const unsigned char* src = reinterpret_cast<const unsigned char*>(Ac + ((size_t)K * S + 1) * NP * NP);
        for (int q = lane; q < Sh::ASZ / Sh::AG; q += 32) cp_async_g<Sh::AG>(cd + q * Sh::AG, src + q * Sh::AG);
      }
      const TI* dsrc = D + (size_t)K * NP * NP;
      if (Sh::DG > 0) {
        const unsigned char* src = reinterpret_cast<const unsigned char*>(dsrc);
        for (int q = lane; q < Sh::DSZ / (Sh::DG > 0 ? Sh::DG : 1); q += 32)
          cp_async_g<(Sh::DG > 0 ? Sh::DG : 4)>(cd + Sh::AB + q * Sh::DG, src + q * Sh::DG);
      } else {
        TI* dd = reinterpret_cast<TI*>(cd + Sh::AB);
        for (int q = lane; q < NP * NP; q += 32) dd[q] = dsrc[q];
      }
    }
  };
  // neighbour indices of this lane's cell in group un (-1: none, or no such cell)
  auto load_nb = [&](int un, int* nb) {
    const int K = un * CPW + hl;
    const bool ok = !first && un < nunits && K < C;
#pragma unroll
    for (int s = 0; s < NF; ++s) nb[s] = ok ? __ldg(nbr + (size_t)K * NF + s) : -1;
  };
  // this lane's columns of the NP rows of cell J's iterate (zeros for J < 0)
  auto load_slab = [&](int J, float (*x)[CPL]) {
    if (J >= 0) {
      const float* p = zo + (size_t)J * NP * R;
#pragma unroll
      for (int j = 0; j < NP; ++j) Cl::ld(p + (size_t)j * R, c0, R, x[j]);
    } else {
#pragma unroll
      for (int j = 0; j < NP; ++j)
#pragma unroll
        for (int c = 0; c < CPL; ++c) x[j][c] = 0.f;
    }
  };

  // Register buffers: t (T), xc (the slab being applied), xn (the next load in flight).
  // Per group the loads are slab 0 .. slab NF-1, then r, then the own iterate zo_K: each is
  // issued one phase before its use (slab s+1 during block s, r during the last block, zo_K
  // while r is added, the next group's slab 0 during the inverse product).
  int nbc[NF], nbn[NF];
  float xc[NP][CPL], xn[NP][CPL];
  load_nb(u, nbc);
  load_unit(u, 0);
  cp_async_commit();
  if (!first) load_slab(nbc[0], xc);
  for (int it = 0; u < nunits; u += nw, ++it) {
    const int st = it & 1;
    const int un = u + nw;
    if (un < nunits) load_unit(un, st ^ 1);
    cp_async_commit();
    load_nb(un, nbn);
    const int K = u * CPW + hl;
    const bool act = K < C;
    float t[NP][CPL];
    if (first && act)
#pragma unroll
      for (int i = 0; i < NP; ++i) Cl::ld(r32 + ((size_t)K * NP + i) * R, c0, R, t[i]);
    cp_async_wait<1>();   // this lane's copies of stage st have landed
    __syncwarp();         // ... and every lane's
    const unsigned char* cb = wbase + ((size_t)st * CPW + hl) * Sh::CS;
    const float* As = reinterpret_cast<const float*>(cb);
    const TI* Ds = reinterpret_cast<const TI*>(cb + Sh::AB);
    if (!first && act) {
#pragma unroll
      for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int c = 0; c < CPL; ++c) t[i][c] = 0.f;
#pragma unroll
      for (int s = 0; s < NF; ++s) {
        if (s + 1 < NF) load_slab(nbc[s + 1], xn);
        else
#pragma unroll
          for (int i = 0; i < NP; ++i) Cl::ld(r32 + ((size_t)K * NP + i) * R, c0, R, xn[i]);
        if (nbc[s] >= 0) {
          const float* Ab = As + s * NP * NP;
#pragma unroll
          for (int i = 0; i < NP; ++i) {
            if (EVEN) {
#pragma unroll
              for (int j = 0; j < NP; j += 2) {
                const float2 a = *reinterpret_cast<const float2*>(Ab + i * NP + j);
#pragma unroll
                for (int c = 0; c < CPL; ++c) {
                  t[i][c] = fmaf(-a.x, xc[j][c], t[i][c]);
                  t[i][c] = fmaf(-a.y, xc[j + 1][c], t[i][c]);
                }
              }
            } else {
#pragma unroll
              for (int j = 0; j < NP; ++j) {
                const float a = Ab[i * NP + j];
#pragma unroll
                for (int c = 0; c < CPL; ++c) t[i][c] = fmaf(-a, xc[j][c], t[i][c]);
              }
            }
          }
        }
#pragma unroll
        for (int j = 0; j < NP; ++j)
#pragma unroll
          for (int c = 0; c < CPL; ++c) xc[j][c] = xn[j][c];
      }
      // xc = r: T = r - sum_s A_s x_s; then xc = zo_K for the damping
#pragma unroll
      for (int i = 0; i < NP; ++i)
#pragma unroll
        for (int c = 0; c < CPL; ++c) t[i][c] += xc[i][c];
#pragma unroll
      for (int i = 0; i < NP; ++i) Cl::ld(zo + ((size_t)K * NP + i) * R, c0, R, xc[i]);
    }
    if (!first) load_slab(nbn[0], xn);   // the next group's first slab
    if (act) {
      // zn = (1 - om) zo + om D^{-1} T
#pragma unroll
      for (int i = 0; i < NP; ++i) {
        float e[CPL];
#pragma unroll
        for (int c = 0; c < CPL; ++c) e[c] = 0.f;
        if (EVEN) {
#pragma unroll
          for (int j = 0; j < NP; j += 2) {
            const float2 d = ld_pair<TI>(Ds + i * NP + j);
#pragma unroll
            for (int c = 0; c < CPL; ++c) {
              e[c] = fmaf(d.x, t[j][c], e[c]);
              e[c] = fmaf(d.y, t[j + 1][c], e[c]);
            }
          }
        } else {
#pragma unroll
          for (int j = 0; j < NP; ++j) {
            const float d = to_f<TI>(Ds[i * NP + j]);
#pragma unroll
            for (int c = 0; c < CPL; ++c) e[c] = fmaf(d, t[j][c], e[c]);
          }
        }
        if (!first) {
#pragma unroll
          for (int c = 0; c < CPL; ++c) e[c] = fmaf(1.f - om, xc[i][c], om * e[c]);
        } else {
#pragma unroll
          for (int c = 0; c < CPL; ++c) e[c] = om * e[c];
        }
        Cl::st(zn + ((size_t)K * NP + i) * R, c0, R, e);
      }
    }
    if (!first)
#pragma unroll
      for (int j = 0; j < NP; ++j)
#pragma unroll
        for (int c = 0; c < CPL; ++c) xc[j][c] = xn[j][c];
#pragma unroll
    for (int s = 0; s < NF; ++s) nbc[s] = nbn[s];
    __syncwarp();   // every lane is done with stage st before the next group refills it
  }
  cp_async_wait<0>();
}

// column blocking of a launch: CPL = 4 with R = 32 (vector accesses), 1 at Np = 20
// (register budget), else 2
int simt_cpl(int np, int R) { return np > 10 ? 1 : R == 32 ? 4 : 2; }

template <typename F>
bool simt_dispatch(int np, int dim, F&& f) {
  switch (np * 10 + dim) {
    case 32: f(std::integral_constant<int, 3>{}, std::integral_constant<int, 5>{}); return true;
    case 62: f(std::integral_constant<int, 6>{}, std::integral_constant<int, 5>{}); return true;
    case 102: f(std::integral_constant<int, 10>{}, std::integral_constant<int, 5>{}); return true;
    case 43: f(std::integral_constant<int, 4>{}, std::integral_constant<int, 7>{}); return true;
    case 103: f(std::integral_constant<int, 10>{}, std::integral_constant<int, 7>{}); return true;
    case 203: f(std::integral_constant<int, 20>{}, std::integral_constant<int, 7>{}); return true;
    default: return false;
  }
}

}  // namespace

size_t msweep_simt_smem(int np, int dim, bool bf16, int R, int wpb) {
  size_t wb = 0;
  const int cpl = simt_cpl(np, R);
  simt_dispatch(np, dim, [&](auto NPc, auto Sc) {
    constexpr int NP = decltype(NPc)::value, S = decltype(Sc)::value;
    if (cpl == 4) wb = bf16 ? SimtShape<NP, S, __nv_bfloat16, 4>::WB : SimtShape<NP, S, float, 4>::WB;
    else if (cpl == 2) wb = bf16 ? SimtShape<NP, S, __nv_bfloat16, 2>::WB : SimtShape<NP, S, float, 2>::WB;
    else wb = bf16 ? SimtShape<NP, S, __nv_bfloat16, 1>::WB : SimtShape<NP, S, float, 1>::WB;
  });
  return wb * wpb;
}

int msweep_simt_units(int np, int R, int C) {
  const int cpw = simt_cpl(np, R);
  return (C + cpw - 1) / cpw;
}

namespace {

// every instantiation a launch can pick for (NP, S, TI, TOUT): f(kernel pointer)
template <int NP, int S, typename TI, typename TOUT, typename F>
void simt_each(F&& f) {
  if constexpr (NP > 10) {
    f(k_msweep_simt<NP, S, TI, TOUT, 1, 0, false>);
  } else {
    f(k_msweep_simt<NP, S, TI, TOUT, 4, 32, true>);
    f(k_msweep_simt<NP, S, TI, TOUT, 2, 0, true>);
    f(k_msweep_simt<NP, S, TI, TOUT, 2, 0, false>);
  }
}

}  // namespace

cudaError_t msweep_simt_prepare(int np, int dim, int smem_optin) {
  cudaError_t err = cudaSuccess;
  auto set = [&](auto kern) {
    const cudaError_t e =
        cudaFuncSetAttribute((const void*)kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_optin);
    if (e != cudaSuccess) err = e;
  };
  const bool ok = simt_dispatch(np, dim, [&](auto NPc, auto Sc) {
    constexpr int NP = decltype(NPc)::value, S = decltype(Sc)::value;
    simt_each<NP, S, float, float>(set);
    simt_each<NP, S, float, double>(set);
    simt_each<NP, S, __nv_bfloat16, float>(set);
    simt_each<NP, S, __nv_bfloat16, double>(set);
  });
  return ok ? err : cudaErrorInvalidValue;
}

int msweep_simt_blocks_per_sm(int np, int dim, bool bf16, int R, int wpb, bool out64) {
  const size_t sm = msweep_simt_smem(np, dim, bf16, R, wpb);
  const int cpl = simt_cpl(np, R);
  int best = 1 << 30;
  auto occ = [&](auto kern) {
    int b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kern, wpb * 32, sm) != cudaSuccess) b = 1;
    best = std::min(best, b);
  };
  // the instantiation (FP32 or FP64 output) a launch of this shape runs
  simt_dispatch(np, dim, [&](auto NPc, auto Sc) {
    constexpr int NP = decltype(NPc)::value, S = decltype(Sc)::value;
    auto one = [&](auto ti, auto to) {
      using TI = decltype(ti);
      using TO = decltype(to);
      if constexpr (NP > 10) {
        occ(k_msweep_simt<NP, S, TI, TO, 1, 0, false>);
      } else {
        if (cpl == 4) occ(k_msweep_simt<NP, S, TI, TO, 4, 32, true>);
        else if (R % 2 == 0) occ(k_msweep_simt<NP, S, TI, TO, 2, 0, true>);
        else occ(k_msweep_simt<NP, S, TI, TO, 2, 0, false>);
      }
    };
    if (bf16) {
      if (out64) one(__nv_bfloat16{}, double{});
      else one(__nv_bfloat16{}, float{});
    } else {
      if (out64) one(float{}, double{});
      else one(float{}, float{});
    }
  });
  return best == (1 << 30) ? 1 : std::max(best, 1);
}

template <typename TI, typename TOUT>
void launch_msweep_simt(int np, int dim, const float* Ac, const TI* D, const int* nbr, int C, int R,
                        const float* r32, const float* zo, TOUT* zn, float om, int first, int wpb, int grid,
                        cudaStream_t s) {
  const size_t sm = msweep_simt_smem(np, dim, std::is_same<TI, __nv_bfloat16>::value, R, wpb);
  const int cpl = simt_cpl(np, R);
  simt_dispatch(np, dim, [&](auto NPc, auto Sc) {
    constexpr int NP = decltype(NPc)::value, S = decltype(Sc)::value;
    if constexpr (NP > 10) {
      k_msweep_simt<NP, S, TI, TOUT, 1, 0, false><<<grid, wpb * 32, sm, s>>>(Ac, D, nbr, C, R, r32, zo, zn, om, first);
    } else {
      if (cpl == 4)
        k_msweep_simt<NP, S, TI, TOUT, 4, 32, true><<<grid, wpb * 32, sm, s>>>(Ac, D, nbr, C, R, r32, zo, zn, om, first);
      else if (R % 2 == 0)
        k_msweep_simt<NP, S, TI, TOUT, 2, 0, true><<<grid, wpb * 32, sm, s>>>(Ac, D, nbr, C, R, r32, zo, zn, om, first);
      else
        k_msweep_simt<NP, S, TI, TOUT, 2, 0, false><<<grid, wpb * 32, sm, s>>>(Ac, D, nbr, C, R, r32, zo, zn, om, first);
    }
  });
}

template void launch_msweep_simt<float, float>(int, int, const float*, const float*, const int*, int, int,
                                               const float*, const float*, float*, float, int, int, int,
                                               cudaStream_t);
template void launch_msweep_simt<float, double>(int, int, const float*, const float*, const int*, int, int,
                                                const float*, const float*, double*, float, int, int, int,
                                                cudaStream_t);
template void launch_msweep_simt<__nv_bfloat16, float>(int, int, const float*, const __nv_bfloat16*, const int*,
                                                       int, int, const float*, const float*, float*, float, int,
                                                       int, int, cudaStream_t);
template void launch_msweep_simt<__nv_bfloat16, double>(int, int, const float*, const __nv_bfloat16*, const int*,
                                                        int, int, const float*, const float*, double*, float, int,
                                                        int, int, cudaStream_t);

}  // namespace kcmg
