// Fused stage kernel for FP32 isothermal Euler in 3D at degrees 5 and 7 (Sec. 2.1-2.3,
// Eq. (eulerIso2d) extended to three momentum components), one thread per line of n nodes for
// all four variables.
//
// It computes what stage_body computes for these classes -- the same operations in the same
// order, so its results are bitwise those of the (line, variable) mapping, which stays on
// stage_body -- with these changes to how the work reaches the SM (measured at 64^3 elements of
// degree 5 / 32^3 of degree 7, ms per RK4 stage: 1.004 / 0.263 before):
//   - shared memory is element-major, [element][variable][SPE] (degree 5: 24 slots of padding
//     per element), so every variable block of a line is a compile-time offset from one base
//     address instead of a multiple of the run-time tile size;
//   - the variables go through the even-odd contraction, the right-hand-side accumulation and
//     the stage update in pairs, in Blackwell's paired FP32 instructions (FFMA2 / FADD2 / FMUL2
//     through __ffma2_rn / __fadd2_rn / __fmul2_rn), each lane rounding exactly as the scalar
//     instruction does (with the layout: 85.7 -> 72.9 warp instructions per DOF, 0.979 / 0.256);
//   - the update issues the global loads of all four variables of a quad before its first
//     store (0.942 / 0.258);
//   - the solve's fields (pointers, scales, RK coefficients) live in shared memory, not in
//     registers, which the line work needs under the 96-register cap (0.939 / 0.232).
// Measured slower and left out: the update's U^n / ACC copied into shared memory by bulk copies,
// a second stage-input slot with the next tile's copy in flight (issued right after the current
// tile's wait: 64^3 0.933 -> 1.066 ms, 32^3 degree 7 0.227 -> 0.305 ms), the next tile's copy
// issued before the update, both quads of a thread's update loaded before either is stored (the
// loads need 64 registers: spills under the cap, 0.933 -> 1.107 ms), ACC alone copied into shared
// memory with the tile on its own barrier and U^n of both quads loaded first (no spills, four
// CTAs per SM still: 0.933 -> 0.982 ms), the neighbour traces staged
// in shared memory by cp.async, neighbour traces inside the tile read from shared memory, register
// caps of 72 and 80 (spills), and two threads per line (one per variable pair).  Also measured
// slower at 64^3 degree 5 (ms per RK4 stage against 0.914-0.917 in the same runs): the stage input
// of the tiles across the upper y and z faces prefetched into L2 by bulk prefetches with the tile
// (0.983; upper z only: 0.979), and an update balanced over the CTA's threads -- each thread one
// x-line of six nodes (1.118: its float2 accesses are 24 bytes apart across a warp) or three
// float2 stripes per variable, consecutive across the warp (1.015, spilling under the cap), and
// the update fused into the z pass, each z-line thread updating its own six nodes from registers
// (no right-hand-side round trip, one barrier less; coalesced 4-byte accesses: 1.190 with the
// loads node by node, 0.961 with all loads of a line before its stores; degree 7: 0.280 vs 0.230).
// The neighbour traces through the read-only path, with or without an L1 evict_last hint,
// measured the same as plain loads (0.922-0.924 ms).
// Phase profile at 64^3 (clock64 at one thread per CTA, all four RK4 stages, cycles per tile of
// four elements): copy wait 3.1k, axis 0 2.2k, axis 1 3.1k, axis 2 3.4k, update 4.1k; with four
// CTAs per SM in these phases the SM issues about half of the cycles.
// The tile arrives as before by bulk copies on an mbarrier (one per element and variable at
// degree 5: 864 contiguous bytes; one per 256-byte z-plane at degree 7), with the same bounded
// wait, failure flag and test switch.
#pragma once

namespace ndg {

// a - b in one paired instruction: a + (-1) b has an exact product and one rounding, so each
// lane equals the scalar subtraction (signed zeros included)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __ffma2_rn(b, make_float2(-1.f, -1.f), a); }
__device__ __forceinline__ float2 dup2(float x) { return make_float2(x, x); }

// Loads of data that a tile reads once (U^n, ACC and stored slopes in the stage update).  At
// degree 7 they take the non-coherent path without allocating in L1, which keeps L1 for the
// neighbour traces (32^3: 0.2340 -> 0.2299 ms per RK4 stage); at degree 5 that measured slower
// (64^3: 0.9129 -> 0.9204 ms), so those stay plain read-only loads.
template <bool NA>
__device__ __forceinline__ float4 ld_stream(const float4* p) {
  if constexpr (NA) {
    float4 r;
    asm("ld.global.nc.L1::no_allocate.v4.f32 {%0, %1, %2, %3}, [%4];"
        : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w)
        : "l"(p));
    return r;
  } else {
    return __ldg(p);
  }
}

template <int N>
struct Euler3dF32Geom {
  static constexpr int n = N + 1;
  static constexpr int L = n * n;        // lines per element along one axis = threads per element
  static constexpr int NPE = n * n * n;  // nodes per element
  static constexpr int NV = 4;
  static constexpr bool PLANE = n == 8;  // degree 7: z-planes 72 slots apart (as StageGeom::PLANE)
  static constexpr int RS = n;
  static constexpr int PS = PLANE ? n * n + 8 : n * n;
  static constexpr int SPE = PLANE ? n * PS : NPE;           // slots of one variable of one element
  // slots of one element, all variables.  Degree 5: 864 + 24 = 888 (= 24 mod 32 banks, the bank
  // offset of the 216-slot element stride of the variable-major layout), so that a warp whose
  // lines straddle two elements meets no more conflicts than there: x-lines as float2
  // conflict-free, y / z lines at most 2-way (864 + 8 would make y-lines 4-way); degree 7: a
  // warp's 32 lines never leave one element.  Both are multiples of 16 bytes (bulk copies).
  static constexpr int ES = NV * SPE + (PLANE ? 0 : 24);
  static constexpr int XW = PLANE ? 4 : 2;  // x-line access width (floats)
  __device__ static __forceinline__ int pad(int node) { return PLANE ? node + 8 * (node / (n * n)) : node; }
};

// the update's loads are non-allocating for the degree-7 class (its SPE) only
template <int SPE>
constexpr bool kDeg7 = SPE == Euler3dF32Geom<7>::SPE;

// D along one line for two variables at once (the even-odd halves of contract_even_odd, even n).
template <int N>
__device__ __forceinline__ void contract_pair(const float2 (&f)[N + 1], float2 (&out)[N + 1], const BasisPairs& B) {
  constexpr int n = N + 1;
  constexpr int H = n / 2;
  static_assert(n % 2 == 0, "even node counts only");
  float2 fe[H], fo[H];
#pragma unroll
  for (int m = 0; m < H; ++m) {
    fe[m] = __fadd2_rn(f[m], f[N - m]);
    fo[m] = sub2(f[m], f[N - m]);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float2 E = __fmul2_rn(B.Ae[i * 4], fo[0]);
    float2 O = __fmul2_rn(B.Bo[i * 4], fe[0]);
#pragma unroll
    for (int m = 1; m < H; ++m) {
      E = __ffma2_rn(B.Ae[i * 4 + m], fo[m], E);
      O = __ffma2_rn(B.Bo[i * 4 + m], fe[m], O);
    }
    out[i] = __fadd2_rn(E, O);
    out[N - i] = sub2(E, O);
  }
}

// Right-hand side of two variables on one line: axis 0 stores, later axes accumulate (with the
// axis scale vs); the face terms lift onto the end nodes.  p0, p1: the variables' line starts.
template <int N, int XW>
__device__ __forceinline__ void accumulate_pair(float* p0, float* p1, int stride, bool vec, bool first, float vs,
                                                float qlo, float qhi, const float2 (&o)[N + 1], float2 flo,
                                                float2 fhi) {
  constexpr int n = N + 1;
  float r0[n], r1[n];
  if (first) {
#pragma unroll
    for (int l = 0; l < n; ++l) {
      float2 r = o[l];
      if (l == 0) r = __ffma2_rn(dup2(qlo), flo, r);
      if (l == N) r = __ffma2_rn(dup2(qhi), fhi, r);
      r0[l] = r.x;
      r1[l] = r.y;
    }
  } else {
    float s0[n], s1[n];
    load_line<n, XW>(p0, stride, vec, s0);
    load_line<n, XW>(p1, stride, vec, s1);
#pragma unroll
    for (int l = 0; l < n; ++l) {
      float2 r = __ffma2_rn(dup2(vs), o[l], make_float2(s0[l], s1[l]));
      if (l == 0) r = __ffma2_rn(dup2(qlo), flo, r);
      if (l == N) r = __ffma2_rn(dup2(qhi), fhi, r);
      r0[l] = r.x;
      r1[l] = r.y;
    }
  }
  store_line<n, XW>(p0, stride, vec, r0);
  store_line<n, XW>(p1, stride, vec, r1);
}

// The fields of the solve that owns the current tile, in shared memory (written by thread 0 when
// the solve changes) instead of registers: the line work keeps the registers.
struct SolveShared {
  const float* uin;  // stage input
  const float* un;   // U^n
  float* acc;        // ACC
  float* uout;       // stage output
  float* kw;         // slope stored by this stage (RK6), or NULL
  const float* halo_lo[3];
  const float* halo_hi[3];
  long long nelem;
  int index, tile_begin;
  unsigned E0, E1, E2;
  float vs[3], qlo[3], qhi[3];
  float c, c2, a_self, bdt, dts;
};

// Stored slopes (RK6): the stage combination of four nodes, W variables at a time (the slopes'
// float4 loads of those variables issued together; node by node, with 4-byte loads between the
// stores, they were serialised: 64^3 RK6 2.19 -> 1.36 ms per stage).  Per node the operations and
// their order are stage_update_node's.
template <int SPE, int W>
__device__ __forceinline__ void stage_update_slopes4(const StageArgs<float>& args, const SolveShared& ss, int si,
                                                     const StagePlan& plan, long long g, long long vstride,
                                                     const float* sr, const float4 (&a)[4], const float4 (&b)[4]) {
  float* acc = ss.acc;
  float* uout = ss.uout;
  float* kw = ss.kw;
  const float a_self = ss.a_self, bdt = ss.bdt;
#pragma unroll
  for (int p = 0; p < 4; p += W) {
    float4 r[W], o[W];
#pragma unroll
    for (int q = 0; q < W; ++q) {
      r[q] = *reinterpret_cast<const float4*>(sr + (p + q) * SPE);
      o[q] = fma4(a_self, r[q], b[p + q]);
    }
    for (int j = 0; j < plan.nread; ++j) {
      const float* kj = static_cast<const float*>(args.solves[si].buf[plan.kread[j]]);
      const float aj = plan.a_read_f[j] * ss.dts;
      float4 kv[W];
#pragma unroll
      for (int q = 0; q < W; ++q)
        kv[q] = ld_stream<kDeg7<SPE>>(reinterpret_cast<const float4*>(kj + (p + q) * vstride + g));
#pragma unroll
      for (int q = 0; q < W; ++q) o[q] = fma4(aj, kv[q], o[q]);
    }
#pragma unroll
    for (int q = 0; q < W; ++q) {
      const long long gv = (p + q) * vstride + g;
      *reinterpret_cast<float4*>(uout + gv) = o[q];
      if (plan.acc_mode == 1) *reinterpret_cast<float4*>(acc + gv) = fma4(bdt, r[q], b[p + q]);
      else if (plan.acc_mode == 2) *reinterpret_cast<float4*>(acc + gv) = fma4(bdt, r[q], a[p + q]);
      if (kw) *reinterpret_cast<float4*>(kw + gv) = r[q];
    }
  }
}

// The update of one quad of all four variables: every global load of the four variables is issued
// before the first store, so their latencies overlap (variable by variable, a store might alias
// the next variable's loads as far as the compiler knows, which would serialise them).  The
// arithmetic per node is stage_update_quad's (stage_update_node's with stored slopes, RK6).
template <int SPE, int SW>
__device__ __forceinline__ void stage_update_quads4(const StageArgs<float>& args, const SolveShared& ss, int si,
                                                    const StagePlan& plan, long long g, long long vstride,
                                                    const float* sr, const float* su) {
  constexpr int NV = 4;
  const float* un = ss.un;
  float* acc = ss.acc;
  float* uout = ss.uout;
  float* kw = ss.kw;
  const float a_self = ss.a_self, bdt = ss.bdt;
  float4 a[NV], b[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    a[v] = b[v] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (plan.acc_mode >= 2) a[v] = ld_stream<kDeg7<SPE>>(reinterpret_cast<const float4*>(acc + v * vstride + g));
    if (plan.acc_mode != 3)
      b[v] = plan.in == kUN ? *reinterpret_cast<const float4*>(su + v * SPE)
                            : ld_stream<kDeg7<SPE>>(reinterpret_cast<const float4*>(un + v * vstride + g));
  }
  if (plan.nread > 0) {
    stage_update_slopes4<SPE, SW>(args, ss, si, plan, g, vstride, sr, a, b);
    return;
  }
#pragma unroll
  for (int v = 0; v < NV; ++v) {
    const float4 r = *reinterpret_cast<const float4*>(sr + v * SPE);
    const long long gv = v * vstride + g;
    const float2 rl = make_float2(r.x, r.y), rh = make_float2(r.z, r.w);
    const float2 al = make_float2(a[v].x, a[v].y), ah = make_float2(a[v].z, a[v].w);
    const float2 bl = make_float2(b[v].x, b[v].y), bh = make_float2(b[v].z, b[v].w);
    if (plan.acc_mode == 3) {
      const float2 ol = __ffma2_rn(dup2(bdt), rl, al), oh = __ffma2_rn(dup2(bdt), rh, ah);
      *reinterpret_cast<float4*>(uout + gv) = make_float4(ol.x, ol.y, oh.x, oh.y);
      continue;
    }
    const float2 ol = __ffma2_rn(dup2(a_self), rl, bl), oh = __ffma2_rn(dup2(a_self), rh, bh);
    *reinterpret_cast<float4*>(uout + gv) = make_float4(ol.x, ol.y, oh.x, oh.y);
    if (plan.acc_mode == 1) {
      const float2 cl = __ffma2_rn(dup2(bdt), rl, bl), ch = __ffma2_rn(dup2(bdt), rh, bh);
      *reinterpret_cast<float4*>(acc + gv) = make_float4(cl.x, cl.y, ch.x, ch.y);
    } else if (plan.acc_mode == 2) {
      const float2 cl = __ffma2_rn(dup2(bdt), rl, al), ch = __ffma2_rn(dup2(bdt), rh, ah);
      *reinterpret_cast<float4*>(acc + gv) = make_float4(cl.x, cl.y, ch.x, ch.y);
    }
    if (kw) *reinterpret_cast<float4*>(kw + gv) = r;
  }
}

template <int N>
__device__ __forceinline__ void euler3d_f32_body(const StageArgs<float>& args) {
  using G = Euler3dF32Geom<N>;
  constexpr int n = G::n, L = G::L, NPE = G::NPE, NV = G::NV, SPE = G::SPE, ES = G::ES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const GroupHeader hdr = *args.hdr;
  const int epb = hdr.epb;
  float* const sU = reinterpret_cast<float*>(smem_raw);  // [epb][ES]: the stage-input tile
  float* const sR = sU + epb * ES;                        // [epb][ES]: the right-hand side
  const size_t moff = ((size_t)2 * epb * ES * sizeof(float) + 15) / 16 * 16;
  unsigned long long* const mbar = reinterpret_cast<unsigned long long*>(smem_raw + moff);  // tile copies
  SolveShared* const sS = reinterpret_cast<SolveShared*>(smem_raw + moff + 16);       // the tile's solve
  const int tid = threadIdx.x;
  const int nthr = blockDim.x;
  const StagePlan& plan = args.plan;
  const int polls = hdr.wait_polls > 0 ? hdr.wait_polls : kBulkWaitPolls;
  if (tid == 0) mbar_init(mbar);
  unsigned phase = 0;
  const int el_t = tid / L;         // this thread's element in the tile
  const int line = tid - el_t * L;  // and its line (along every axis in turn)
  const bool need_un = plan.in != kUN && plan.acc_mode != 3;
  const bool need_acc = plan.acc_mode >= 2;

  // The tile starting at element e0 (cnt elements) of the current solve into sU, and its U^n / ACC
  // into L2; called by warp 0.
  auto issue_tile = [&](long long e0, int cnt, long long vstride) {
    fence_proxy_async_smem();  // this CTA's earlier reads of sU before the asynchronous writes
    const unsigned bytes = (unsigned)(cnt * NPE * sizeof(float));
    if (tid == 0) mbar_expect_tx(mbar, bytes * NV);
    if (!hdr.stall_copies) {
      __syncwarp();
      const float* src = sS->uin + e0 * NPE;
      if constexpr (G::PLANE) {
        constexpr int per = NV * n;  // copies per element: one per variable and z-plane
        for (int k = tid; k < cnt * per; k += 32) {
          const int el = k / per, r = k - el * per, v = r / n, z = r - v * n;
          bulk_copy(sU + el * ES + v * SPE + z * G::PS, src + v * vstride + el * NPE + z * (n * n),
                    n * n * sizeof(float), mbar);
        }
      } else {
        for (int k = tid; k < cnt * NV; k += 32) {
          const int el = k / NV, v = k - el * NV;
          bulk_copy(sU + el * ES + v * SPE, src + v * vstride + el * NPE, NPE * sizeof(float), mbar);
        }
      }
    }
    if (tid == 0) {
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        if (need_un) bulk_prefetch_l2(sS->un + v * vstride + e0 * NPE, bytes);
        if (need_acc) bulk_prefetch_l2(sS->acc + v * vstride + e0 * NPE, bytes);
      }
    }
  };

  int cur = -1;  // the solve whose fields sS holds
  for (int tile = blockIdx.x; tile < hdr.ntiles; tile += gridDim.x) {
    const int si = hdr.nsolves > 1 ? find_solve(args.solves, hdr.nsolves, tile) : 0;
    if (si != cur) {
      // a new solve (the same for every thread): thread 0 writes its fields; every reader of the
      // previous ones finished before the closing barrier of the previous tile
      if (tid == 0) {
        SolveRegs<3, float> R;
        R.load(args.solves + si, si, plan);
        SolveShared& w = *sS;
        w.uin = R.uin, w.un = R.un, w.acc = R.acc, w.uout = R.uout, w.kw = R.kw;
#pragma unroll
        for (int x = 0; x < 3; ++x) {
          w.halo_lo[x] = R.halo_lo[x], w.halo_hi[x] = R.halo_hi[x];
          w.vs[x] = R.vs[x], w.qlo[x] = R.qlo[x], w.qhi[x] = R.qhi[x];
        }
        w.nelem = R.nelem, w.index = si, w.tile_begin = R.tile_begin;
        w.E0 = R.E0, w.E1 = R.E1, w.E2 = R.E2;
        w.c = R.c, w.c2 = R.c2, w.a_self = R.a_self, w.bdt = R.bdt, w.dts = R.dts;
      }
      cur = si;
      __syncthreads();
    }
    const long long nelem = sS->nelem;
    const long long e0 = (long long)(tile - sS->tile_begin) * epb;
    const int cnt = (int)min((long long)epb, nelem - e0);
    const long long vstride = nelem * NPE;

    // ---- 1. the tile by bulk copies (warp 0, after lane 0 has armed the barrier), and the
    //         update's U^n / ACC prefetched into L2 ----
    if (tid < 32) issue_tile(e0, cnt, vstride);
    const bool ok = mbar_wait(mbar, phase, polls);
    if (!__syncthreads_and(ok)) {
      // the copies did not land in time: flag the launch for the host, give the copies in flight
      // one more bounded wait, and leave
      if (tid == 0) flag_failure(args);
      mbar_wait(mbar, phase, polls);
      return;
    }
    phase ^= 1u;

    // ---- 2. volume + surface terms, axis by axis ----
    const ElemXYZ exyz = elem_xyz((unsigned)(e0 + el_t), sS->E0, sS->E1);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      if (el_t < cnt) {
        int pbase, pstride, ubase, ustride;
        line_geometry<n, G::RS, G::PS>(a, line, pbase, pstride, ubase, ustride);
        const float* sUe = sU + el_t * ES + pbase;
        float* sRe = sR + el_t * ES + pbase;
        const bool VX = a == 0;  // x-lines: contiguous, read and written as float2 / float4
        // exterior traces (node N of the low neighbour, node 0 of the high one): from the stage
        // input in global memory (read-only during the stage), or from a partition halo
        float xlo[NV], xhi[NV];
        {
          const float* hlo = sS->halo_lo[a];
          const float* hhi = sS->halo_hi[a];
          const float* uin = sS->uin;
          const LineTrace t = line_trace<L>(a, (unsigned)(e0 + el_t), exyz, line, sS->E0, sS->E1, sS->E2,
                                            hlo != nullptr, hhi != nullptr);
          const float* plo = uin + t.elo * NPE + ubase + N * ustride;
          const float* phi = uin + t.ehi * NPE + ubase;
          if (!hlo && !hhi) {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              xlo[v] = plo[v * vstride];
              xhi[v] = phi[v * vstride];
            }
          } else {
#pragma unroll
            for (int v = 0; v < NV; ++v) {
              if (t.lo_halo) xlo[v] = hlo[v * t.hvs + t.hoff];
              else xlo[v] = plo[v * vstride];
              if (t.hi_halo) xhi[v] = hhi[v * t.hvs + t.hoff];
              else xhi[v] = phi[v * vstride];
            }
          }
        }
        const float c2 = sS->c2, cs = sS->c;
        // density, normal momentum and normal velocity along the line; LLF alpha at both faces
        float rho[n], ma[n], ua[n];
        load_line<n, G::XW>(sUe, pstride, VX, rho);
        load_line<n, G::XW>(sUe + (1 + a) * SPE, pstride, VX, ma);
#pragma unroll
        for (int l = 0; l < n; ++l) ua[l] = ratio(ma[l], rho[l]);
        const float un0 = ua[0], unN = ua[N];
        const float unlo = ratio(xlo[1 + a], xlo[0]);
        const float unhi = ratio(xhi[1 + a], xhi[0]);
        const float alo = fmaxf(fabsf(unlo), fabsf(un0)) + cs;
        const float ahi = fmaxf(fabsf(unN), fabsf(unhi)) + cs;
        const float vs = sS->vs[a], qlo = sS->qlo[a], qhi = sS->qhi[a];
        {
          // variables 0 and 1 + a: fluxes m_a and m_a u_a + c^2 rho
          float2 f[n], o[n];
#pragma unroll
          for (int l = 0; l < n; ++l) f[l] = make_float2(ma[l], fmaf(ma[l], ua[l], c2 * rho[l]));
          contract_pair<N>(f, o, args.bp);
          const float fxlo1 = fmaf(xlo[1 + a], unlo, c2 * xlo[0]);
          const float fxhi1 = fmaf(xhi[1 + a], unhi, c2 * xhi[0]);
          // (Fhat_lo - F(U_0)) and (F(U_N) - Fhat_hi) with the 1/2 carried by qlo / qhi
          const float2 flo = make_float2(fmaf(-alo, rho[0] - xlo[0], xlo[1 + a] - f[0].x),
                                         fmaf(-alo, ma[0] - xlo[1 + a], fxlo1 - f[0].y));
          const float2 fhi = make_float2(fmaf(ahi, xhi[0] - rho[N], f[N].x - xhi[1 + a]),
                                         fmaf(ahi, xhi[1 + a] - ma[N], f[N].y - fxhi1));
          accumulate_pair<N, G::XW>(sRe, sRe + (1 + a) * SPE, pstride, VX, a == 0, vs, qlo, qhi, o, flo, fhi);
        }
        {
          // the transverse momenta b1 < b2: fluxes m_b u_a
          const int b1 = a == 0 ? 2 : 1, b2 = a == 2 ? 2 : 3;
          float m1[n], m2[n];
          load_line<n, G::XW>(sUe + b1 * SPE, pstride, VX, m1);
          load_line<n, G::XW>(sUe + b2 * SPE, pstride, VX, m2);
          float2 f[n], o[n];
#pragma unroll
          for (int l = 0; l < n; ++l) f[l] = make_float2(mul_rn(m1[l], ua[l]), mul_rn(m2[l], ua[l]));
          contract_pair<N>(f, o, args.bp);
          const float fxlo1 = mul_rn(xlo[b1], unlo), fxhi1 = mul_rn(xhi[b1], unhi);
          const float fxlo2 = mul_rn(xlo[b2], unlo), fxhi2 = mul_rn(xhi[b2], unhi);
          const float2 flo = make_float2(fmaf(-alo, m1[0] - xlo[b1], fxlo1 - f[0].x),
                                         fmaf(-alo, m2[0] - xlo[b2], fxlo2 - f[0].y));
          const float2 fhi = make_float2(fmaf(ahi, xhi[b1] - m1[N], f[N].x - fxhi1),
                                         fmaf(ahi, xhi[b2] - m2[N], f[N].y - fxhi2));
          accumulate_pair<N, G::XW>(sRe + b1 * SPE, sRe + b2 * SPE, pstride, VX, a == 0, vs, qlo, qhi, o, flo, fhi);
        }
      }
      __syncthreads();
    }

    // ---- 3. Runge-Kutta stage update: four consecutive nodes of every variable per step ----
    // stored slopes (RK6) two variables at a time at degree 5, one at degree 7, where wider
    // batches cost the RK4 stages registers (RK4 / RK6 ms per stage, widths 1, 2, 4: degree 5 at
    // 64^3 0.930 / 1.630, 0.914 / 1.364, 0.915 / 1.350; degree 7 at 32^3 0.2327 / 0.387, 0.2361 /
    // 0.375, 0.2613 / 0.415)
    constexpr int SLOPE_W = N == 7 ? 1 : 2;
    const int quads = cnt * NPE / 4;
    for (int q = tid; q < quads; q += nthr) {
      const int el = q / (NPE / 4);
      const int node = 4 * (q - el * (NPE / 4));
      const int sl = el * ES + G::pad(node);
      stage_update_quads4<SPE, SLOPE_W>(args, *sS, si, plan, e0 * NPE + 4 * q, vstride, sR + sl, sU + sl);
    }
    __syncthreads();
  }
}

// Shared memory of one CTA: the tile and the right-hand side, the mbarrier, the solve's fields.
template <int N>
constexpr size_t euler3d_f32_smem(int epb) {
  return ((size_t)2 * epb * Euler3dF32Geom<N>::ES * sizeof(float) + 15) / 16 * 16 + 16 +
         (sizeof(SolveShared) + 15) / 16 * 16;
}

}  // namespace ndg
