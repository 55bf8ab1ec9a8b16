// sweep_x.cu -- the x sweep of one split step: the H1 substep (Eq. eq1,
// exact pointwise solution) fused into the Crank-Nicolson solve of H2
// (Eq. eq2, discretised as Eq. eqD.9 with the coefficients of Eqs.
// eqD.11/eq5), with the pending imaginary-time renormalisation applied as
// the state is read.
//
// x lines are contiguous: the warp copies 32*V rows x (C + 1) points of a
// chunk cooperatively (coalesced 8- or 16-byte copies) into rows padded to
// an odd number of 16-byte units; each lane then walks its own V rows with
// 16-byte shared loads (conflict-free) and the results go back through the
// same slot for coalesced stores.  The solver and the ring are described in
// sweep_common.cuh.
#include "sweep_common.cuh"
#include "tma.cuh"

namespace rotgp {


template <class T, int V, int C, bool IMAG, bool VEC16>
__global__ void __launch_bounds__(128) k_sweep_x(const stream_args a) {
  using E = cpx<T>;
  constexpr bool F32 = sizeof(T) == 4;
  constexpr int EP = (F32 && VEC16) ? 2 : 1;          // points per copy
  constexpr int PITCH = F32 ? C + 2 : C + 1;           // odd number of 16-byte units
  constexpr int ROWS = 32 * V;
  constexpr int SLOT = ROWS * PITCH;
  constexpr int LPR = (C + 1 + EP - 1) / EP;           // copies per row (chunk + 1 point)
  constexpr int SPR = C / EP;                          // stores per row
  static_assert(LPR * EP <= PITCH, "row pitch too small");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int R = a.ring;
  if (R < 3 || R > 4 ||
      dynamic_smem_bytes() < (blockDim.x >> 5) * (unsigned)(R * SLOT) * (unsigned)sizeof(E)) {
    if (threadIdx.x == 0) atomicOr(a.flags, 2);
    return;
  }
  E* ring = reinterpret_cast<E*>(smem_raw) + (size_t)wib * R * SLOT;
  const long long nrows = a.nlines;
  const long long ngroups = (nrows + ROWS - 1) / ROWS;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  if (wg >= ngroups * a.nseg) return;  // whole warp; no block barrier below
  const long long g = wg % ngroups;
  const int sg = (int)(wg / ngroups);
  const long long row0 = g * ROWS;
  const int N = a.len, nch = (N + C - 1) / C, lt = a.lt;
  const int qo0 = sg * a.seg_chunks, qo1 = min(nch, qo0 + a.seg_chunks);
  const int qa = max(0, qo0 - a.warm), qb = min(nch, qo1 + 1);
  const E* in = static_cast<const E*>(a.in);
  E* out = static_cast<E*>(a.out);

  const coef5<T>* crow[V];
  coef5<T> cinf[V];
  T vyz[V];
#pragma unroll
  for (int v = 0; v < V; ++v) {
    const long long rr = row0 + lane + 32 * v;
    const bool act = rr < nrows;
    const int j = act ? (int)(rr % a.ny) : 0;
    const int k = act ? (int)(rr / a.ny) : 0;
    crow[v] = static_cast<const coef5<T>*>(a.coef) + (size_t)j * (lt + 1);
    cinf[v] = crow[v][lt];
    const T y = (T)(a.y0 + (double)j * a.hy), z = (T)(a.z0 + (double)k * a.hz);
    vyz[v] = (T)a.hnu2 * y * y + (T)a.hlam2 * z * z;
  }
  const T s = (T)(*a.scale), hg2 = (T)a.hgam2, gg = (T)a.g, dt = (T)a.dt;
  const T xs = (T)a.x0, hx = (T)a.hx;
  // psi at position p of lane row v, scaled and advanced by H1
  auto h1 = [&](E psi, int p, int v) -> E {
    psi = s * psi;
    const T x = xs + (T)p * hx;
    const T en = hg2 * x * x + vyz[v] + gg * abs2(psi);
    if (IMAG) {
      return exp_t(-dt * en) * psi;
    } else {
      T c1, s1;
      rot_t(dt * en, &c1, &s1);
      return mk<T>(fma(c1, psi.x, fma(s1, psi.y, psi.x)), fma(c1, psi.y, fma(-s1, psi.x, psi.y)));
    }
  };
  auto slot = [&](int q) { return ring + (size_t)(q % R) * SLOT; };
  auto issue = [&](int q) {
    if (q < qb) {
      E* sl = slot(q);
      for (int t = lane; t < ROWS * LPR; t += 32) {
        const int row = t / LPR, col = t % LPR;
        const int p = q * C + col * EP;
        const long long rr = row0 + row;
        E* dst = sl + row * PITCH + col * EP;
        if (rr < nrows && p < N) {
          cp_async<EP * sizeof(E)>(dst, in + rr * N + p);
        } else {
#pragma unroll
          for (int e = 0; e < EP; ++e) dst[e] = zero<T>();
        }
      }
    }
    cp_async_commit();
  };
  // lane-row access to points 2k, 2k+1 through one 16-byte shared access
  // (float) or two (double)
  auto load2 = [&](const E* rp, int k, E& e0, E& e1) {
    if (F32) {
      const float4 t = reinterpret_cast<const float4*>(rp)[k];
      e0 = mk<T>((T)t.x, (T)t.y);
      e1 = mk<T>((T)t.z, (T)t.w);
    } else {
      e0 = rp[2 * k];
      e1 = rp[2 * k + 1];
    }
  };
  auto store2 = [&](E* rp, int k, E e0, E e1) {
    if (F32) {
      reinterpret_cast<float4*>(rp)[k] =
          make_float4((float)e0.x, (float)e0.y, (float)e1.x, (float)e1.y);
    } else {
      rp[2 * k] = e0;
      rp[2 * k + 1] = e1;
    }
  };
  // real time: psi at position p scaled and held as value + H1 increment
  auto h1p = [&](E psi, int p, int v) -> hpt<T> {
    psi = s * psi;
    const T x = xs + (T)p * hx;
    const T en = hg2 * x * x + vyz[v] + gg * abs2(psi);
    T c1, s1;
    rot_t(dt * en, &c1, &s1);
    return rot_inc(psi, c1, s1);
  };
  // real-time forward sweep over one chunk (the centre point of every step
  // enters as value + increment, fwd_inc)
  auto forward_rt = [&](auto fast_tag, E* s0, int p0, E (&pm)[V], E (&d)[V]) {
    constexpr bool FAST = decltype(fast_tag)::value;
    hpt<T> c0[V], c1[V];
#pragma unroll
    for (int v = 0; v < V; ++v) {
      E r0, r1;
      load2(s0 + (lane + 32 * v) * PITCH, 0, r0, r1);
      c0[v] = h1p(r0, p0, v);
      c1[v] = h1p(r1, p0 + 1, v);
    }
#pragma unroll(unroll_of<C / 2>::value)
    for (int k = 0; k < C / 2; ++k) {
      const int p = p0 + 2 * k;
      hpt<T> n0[V], n1[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        if (k + 1 < C / 2) {
          E r0, r1;
          load2(s0 + (lane + 32 * v) * PITCH, k + 1, r0, r1);
          n0[v] = h1p(r0, p + 2, v);
          n1[v] = h1p(r1, p + 3, v);
        } else {
          n0[v] = h1p(s0[(lane + 32 * v) * PITCH + C], p + 2, v);
          n1[v] = {zero<T>(), zero<T>()};
        }
        const E w1 = hw(c1[v]);
        d[v] = fwd_inc(coef_at<T, FAST>(crow[v], cinf[v], p, lt), pm[v], c0[v], w1, d[v]);
        const E e0 = d[v];
        d[v] = fwd_inc(coef_at<T, FAST>(crow[v], cinf[v], p + 1, lt), hw(c0[v]), c1[v],
                       hw(n0[v]), d[v]);
        store2(s0 + (lane + 32 * v) * PITCH, k, e0, d[v]);
        pm[v] = w1;
        c0[v] = n0[v];
        c1[v] = n1[v];
      }
    }
  };
  // forward sweep over one chunk of the lane's V rows (psi -> d' in place)
  auto forward = [&](auto fast_tag, E* s0, int p0, E (&pm)[V], E (&d)[V]) {
    if constexpr (!IMAG) {
      forward_rt(fast_tag, s0, p0, pm, d);
    } else {
      constexpr bool FAST = decltype(fast_tag)::value;
      E c0[V], c1[V];
#pragma unroll
      for (int v = 0; v < V; ++v) {
        load2(s0 + (lane + 32 * v) * PITCH, 0, c0[v], c1[v]);
        c0[v] = h1(c0[v], p0, v);
        c1[v] = h1(c1[v], p0 + 1, v);
      }
#pragma unroll(unroll_of<C / 2>::value)
      for (int k = 0; k < C / 2; ++k) {
        const int p = p0 + 2 * k;
        E n0[V], n1[V];
#pragma unroll
        for (int v = 0; v < V; ++v) {
          if (k + 1 < C / 2) {
            load2(s0 + (lane + 32 * v) * PITCH, k + 1, n0[v], n1[v]);
            n0[v] = h1(n0[v], p + 2, v);
            n1[v] = h1(n1[v], p + 3, v);
          } else {
            n0[v] = h1(s0[(lane + 32 * v) * PITCH + C], p + 2, v);
            n1[v] = zero<T>();
          }
          d[v] = fwd(coef_at<T, FAST>(crow[v], cinf[v], p, lt), pm[v], c0[v], c1[v], d[v]);
          const E e0 = d[v];
          d[v] = fwd(coef_at<T, FAST>(crow[v], cinf[v], p + 1, lt), c0[v], c1[v], n0[v], d[v]);
          store2(s0 + (lane + 32 * v) * PITCH, k, e0, d[v]);
          pm[v] = c1[v];
          c0[v] = n0[v];
          c1[v] = n1[v];
        }
      }
    }
  };
  // back substitution over chunk slot sp (positions p0..p0+C-1), x carried in
  auto backward = [&](auto fast_tag, E* sp, int p0, E (&x)[V]) {
    constexpr bool FAST = decltype(fast_tag)::value;
#pragma unroll(unroll_of<C / 2>::value)
    for (int k = C / 2 - 1; k >= 0; --k) {
      const int p = p0 + 2 * k;
#pragma unroll
      for (int v = 0; v < V; ++v) {
        E d0, d1;
        load2(sp + (lane + 32 * v) * PITCH, k, d0, d1);
        if (FAST || p + 1 < N) x[v] = bwd(coef_at<T, FAST>(crow[v], cinf[v], p + 1, lt).be, x[v], d1);
        const E e1 = x[v];
        if (FAST || p < N) x[v] = bwd(coef_at<T, FAST>(crow[v], cinf[v], p, lt).be, x[v], d0);
        store2(sp + (lane + 32 * v) * PITCH, k, x[v], e1);
      }
    }
  };

  for (int i = 0; i < R - 1; ++i) issue(qa + i);
  E pm[V], d[V];
#pragma unroll
  for (int v = 0; v < V; ++v) pm[v] = d[v] = zero<T>();
  for (int q = qa; q <= qb; ++q) {
    if (q < qb) {
      ring_wait(R);
      __syncwarp();
      if (q * C >= lt && (q + 1) * C <= N)
        forward(bool_tag<true>{}, slot(q), q * C, pm, d);
      else
        forward(bool_tag<false>{}, slot(q), q * C, pm, d);
    }
    const int qq = q - 1;
    if (qq >= qo0 && qq < qo1) {
      E x[V];
#pragma unroll
      for (int v = 0; v < V; ++v) x[v] = zero<T>();
      const int la = min(a.halo, N - q * C);
      const E* sq = slot(q);
      for (int h = la - 1; h >= 0; --h) {
#pragma unroll
        for (int v = 0; v < V; ++v) {
          const E be = crow[v][min(q * C + h, lt)].be;
          x[v] = bwd(be, x[v], sq[(lane + 32 * v) * PITCH + h]);
        }
      }
      E* sp = slot(qq);
      if (qq * C >= lt && q * C <= N)
        backward(bool_tag<true>{}, sp, qq * C, x);
      else
        backward(bool_tag<false>{}, sp, qq * C, x);
      __syncwarp();
      // coalesced store of chunk qq
#pragma unroll
      for (int i = 0; i < ROWS * SPR / 32; ++i) {
        const int t = i * 32 + lane;
        const int row = t / SPR, col = t % SPR;
        const int p = qq * C + col * EP;
        const long long rr = row0 + row;
        if (rr < nrows && p < N) {
          const E* src = sp + row * PITCH + col * EP;
          if (EP == 2)
            *reinterpret_cast<float4*>(out + rr * N + p) = *reinterpret_cast<const float4*>(src);
          else
            out[rr * N + p] = *src;
        }
      }
    }
    __syncwarp();
    issue(q + R - 1);
  }
  cp_async_wait<0>();
}

// Complex float, two rows per lane (rows lane and lane + 32): the same
// pipeline with the two rows in split form, so that H1 and the recurrences
// run as packed FP32x2 arithmetic (sweep_common.cuh).  The ring keeps each
// row interleaved (the cooperative copies and stores need that); rows are
// split on the 16-byte shared loads and joined on the stores.
//
// TMA = true: each chunk (64 rows x C + 2 points, exactly a ring slot) is
// one 2-D TMA box issued by lane 0 on a per-slot barrier, instead of the
// lanes' cooperative copies (needs 16-byte rows, VEC16).
template <int C, bool IMAG, bool VEC16, bool TMA, int RING>
__global__ void __launch_bounds__(128) k_sweep_x2(const __grid_constant__ CUtensorMap map,
                                                  const stream_args a) {
  using E = cpx<float>;
  constexpr int R = RING;  // ring slots (3 or 4), compile-time for cheap slot indices
  constexpr int EP = VEC16 ? 2 : 1;
  constexpr int PITCH = C + 2;                 // odd number of 16-byte units
  constexpr int ROWS = 64;
  constexpr int SLOT = ROWS * PITCH;
  constexpr int LPR = (C + 1 + EP - 1) / EP;
  constexpr int SPR = C / EP;
  static_assert(LPR * EP <= PITCH, "row pitch too small");
  static_assert(!TMA || (VEC16 && (SLOT * 8) % 128 == 0), "TMA slots");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[TMA ? 4 * 4 : 1];  // [warp][slot]
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const unsigned pad = TMA ? 128 : 0;  // TMA destinations start on 128 bytes
  if (a.ring != R || (TMA && blockDim.x > 128) ||
      dynamic_smem_bytes() <
          (blockDim.x >> 5) * (unsigned)(R * SLOT) * (unsigned)sizeof(E) + pad) {
    if (threadIdx.x == 0) atomicOr(a.flags, 2);
    return;
  }
  unsigned char* sbase =
      TMA ? smem_raw + ((128 - (smem_addr(smem_raw) & 127)) & 127) : smem_raw;
  E* ring = reinterpret_cast<E*>(sbase) + (size_t)wib * R * SLOT;
  uint64_t* bar = bars + (TMA ? wib * 4 : 0);
  const long long nrows = a.nlines;
  const long long ngroups = (nrows + ROWS - 1) / ROWS;
  const long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + wib;
  if (wg >= ngroups * a.nseg) return;  // whole warp; no block barrier below
  const long long g = wg % ngroups;
  const int sg = (int)(wg / ngroups);
  const long long row0 = g * ROWS;
  const int N = a.len, nch = (N + C - 1) / C, lt = a.lt;
  const int qo0 = sg * a.seg_chunks, qo1 = min(nch, qo0 + a.seg_chunks);
  const int qa = max(0, qo0 - a.warm), qb = min(nch, qo1 + 1);
  const E* in = static_cast<const E*>(a.in);
  E* out = static_cast<E*>(a.out);

  const coef5<float>* crow[2];
  float vyz[2];
#pragma unroll
  for (int v = 0; v < 2; ++v) {
    const long long rr = row0 + lane + 32 * v;
    const bool act = rr < nrows;
    const int j = act ? (int)(rr % a.ny) : 0;
    const int k = act ? (int)(rr / a.ny) : 0;
    crow[v] = static_cast<const coef5<float>*>(a.coef) + (size_t)j * (lt + 1);
    const float y = (float)(a.y0 + (double)j * a.hy), z = (float)(a.z0 + (double)k * a.hz);
    vyz[v] = (float)a.hnu2 * y * y + (float)a.hlam2 * z * z;
  }
  const coef2 cf = make_coef2(crow[0][lt], crow[1][lt]);
  const float s = (float)(*a.scale), hg2 = (float)a.hgam2, dt = (float)a.dt;
  const float2 S2 = make_float2(s, s), G2 = make_float2((float)a.g, (float)a.g);
  const float2 VYZ = make_float2(vyz[0], vyz[1]);
  const float xs = (float)a.x0, hx = (float)a.hx;
  // psi of both rows at position p: scaled and advanced by H1
  auto h1 = [&](c2 v, int p) -> c2 {
    v.re = __fmul2_rn(S2, v.re);
    v.im = __fmul2_rn(S2, v.im);
    const float x = xs + (float)p * hx;
    const float vx = hg2 * x * x;
    const float2 dens = __ffma2_rn(v.im, v.im, __fmul2_rn(v.re, v.re));
    const float2 en = __ffma2_rn(G2, dens, __fadd2_rn(VYZ, make_float2(vx, vx)));
    if (IMAG) {
      const float2 f = make_float2(__expf(-dt * en.x), __expf(-dt * en.y));
      v.re = __fmul2_rn(f, v.re);
      v.im = __fmul2_rn(f, v.im);
    }
    return v;
  };
  // real time: both rows' psi at p scaled, and the H1 increment dl (see hpt)
  auto h1_inc = [&](c2& v, int p) -> c2 {
    v.re = __fmul2_rn(S2, v.re);
    v.im = __fmul2_rn(S2, v.im);
    const float x = xs + (float)p * hx;
    const float vx = hg2 * x * x;
    const float2 dens = __ffma2_rn(v.im, v.im, __fmul2_rn(v.re, v.re));
    const float2 en = __ffma2_rn(G2, dens, __fadd2_rn(VYZ, make_float2(vx, vx)));
    float2 s1, c1;
    rot_t(dt * en.x, &c1.x, &s1.x);
    rot_t(dt * en.y, &c1.y, &s1.y);
    c2 dl;
    dl.re = __ffma2_rn(c1, v.re, __fmul2_rn(s1, v.im));
    dl.im = __ffma2_rn(c1, v.im, __fmul2_rn(make_float2(-s1.x, -s1.y), v.re));
    return dl;
  };
  auto slot = [&](int q) { return ring + (size_t)((q - qa) % R) * SLOT; };
  auto issue = [&](int q) {
    if (TMA) {
      if (q < qb && lane == 0) {
        const int sl = (q - qa) % R;
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_expect_tx(&bar[sl], (unsigned)(SLOT * sizeof(E)));
        tma_load_2d(ring + (size_t)sl * SLOT, &map, 2 * q * C, (int)row0, &bar[sl]);
      }
      return;
    }
    if (q < qb) {
      E* sl = slot(q);
      for (int t = lane; t < ROWS * LPR; t += 32) {
        const int row = t / LPR, col = t % LPR;
        const int p = q * C + col * EP;
        const long long rr = row0 + row;
        E* dst = sl + row * PITCH + col * EP;
        if (rr < nrows && p < N) {
          cp_async<EP * sizeof(E)>(dst, in + rr * N + p);
        } else {
#pragma unroll
          for (int e = 0; e < EP; ++e) dst[e] = zero<float>();
        }
      }
    }
    cp_async_commit();
  };
  // points 2k, 2k+1 of both lane rows, split; and the inverse
  auto load_pair = [&](const E* sl, int k, c2& e0, c2& e1) {
    const float4 u = reinterpret_cast<const float4*>(sl + lane * PITCH)[k];
    const float4 w = reinterpret_cast<const float4*>(sl + (lane + 32) * PITCH)[k];
    e0.re = make_float2(u.x, w.x);
    e0.im = make_float2(u.y, w.y);
    e1.re = make_float2(u.z, w.z);
    e1.im = make_float2(u.w, w.w);
  };
  auto store_pair = [&](E* sl, int k, const c2& e0, const c2& e1) {
    reinterpret_cast<float4*>(sl + lane * PITCH)[k] = make_float4(e0.re.x, e0.im.x, e1.re.x, e1.im.x);
    reinterpret_cast<float4*>(sl + (lane + 32) * PITCH)[k] =
        make_float4(e0.re.y, e0.im.y, e1.re.y, e1.im.y);
  };
  auto coef_p = [&](auto fast_tag, int p) -> coef2 {
    if (decltype(fast_tag)::value) return cf;
    const int i = min(p, lt);
    return make_coef2(crow[0][i], crow[1][i]);
  };
  // forward sweep over one chunk: stage the lane's two rows (and the next
  // point) in registers, advance them by H1, solve, write d' back
  auto forward = [&](auto fast_tag, E* s0, int p0, c2& pm, c2& d) {
    c2 w[C + 1];
#pragma unroll
    for (int k = 0; k < C / 2; ++k) load_pair(s0, k, w[2 * k], w[2 * k + 1]);
    w[C].re = make_float2(s0[lane * PITCH + C].x, s0[(lane + 32) * PITCH + C].x);
    w[C].im = make_float2(s0[lane * PITCH + C].y, s0[(lane + 32) * PITCH + C].y);
    if (IMAG) {
#pragma unroll
      for (int r = 0; r <= C; ++r) w[r] = h1(w[r], p0 + r);
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const c2 pc = w[r];
        d = fwd2(coef_p(fast_tag, p0 + r), pm, pc, w[r + 1], d);
        pm = pc;
        w[r] = d;
      }
    } else {
      // the centre point as value + increment, its neighbours rounded
      c2 dl = h1_inc(w[0], p0);
#pragma unroll
      for (int r = 0; r < C; ++r) {
        const c2 dn = h1_inc(w[r + 1], p0 + r + 1);
        c2 pn;
        pn.re = __fadd2_rn(w[r + 1].re, dn.re);
        pn.im = __fadd2_rn(w[r + 1].im, dn.im);
        c2 pc;
        pc.re = __fadd2_rn(w[r].re, dl.re);
        pc.im = __fadd2_rn(w[r].im, dl.im);
        d = fwd2_inc(coef_p(fast_tag, p0 + r), pm, w[r], dl, pn, d);
        pm = pc;
        w[r] = d;
        dl = dn;
      }
    }
#pragma unroll
    for (int k = 0; k < C / 2; ++k) store_pair(s0, k, w[2 * k], w[2 * k + 1]);
  };
  // back substitution over chunk slot sp (positions p0..p0+C-1), x carried in
  auto backward = [&](auto fast_tag, E* sp, int p0, c2& x) {
    constexpr bool FAST = decltype(fast_tag)::value;
    c2 w[C];
#pragma unroll
    for (int k = 0; k < C / 2; ++k) load_pair(sp, k, w[2 * k], w[2 * k + 1]);
#pragma unroll
    for (int r = C - 1; r >= 0; --r) {
      if (FAST || p0 + r < N) x = bwd2(coef_p(fast_tag, p0 + r).be, x, w[r]);
      w[r] = x;
    }
#pragma unroll
    for (int k = 0; k < C / 2; ++k) store_pair(sp, k, w[2 * k], w[2 * k + 1]);
  };

  if (TMA) {
    if (lane == 0) {
      for (int i = 0; i < R; ++i) mbar_init(&bar[i], 1);
      mbar_fence_init();
    }
    __syncwarp();
  }
  for (int i = 0; i < R - 1; ++i) issue(qa + i);
  c2 pm = zero2(), d = zero2();
  for (int q = qa; q <= qb; ++q) {
    if (q < qb) {
      if (TMA) {
        if (!__all_sync(0xffffffffu,
                        mbar_wait(&bar[(q - qa) % R], (unsigned)(((q - qa) / R) & 1)))) {
          // a TMA load never landed: let the other loads in flight land, report, stop
          for (int r = q + 1; r < min(q + R - 1, qb); ++r)
            mbar_wait(&bar[(r - qa) % R], (unsigned)(((r - qa) / R) & 1));
          if (lane == 0) atomicOr(a.flags, 4);
          return;
        }
      } else if (R == 3) {
        cp_async_wait<1>();
      } else {
        cp_async_wait<2>();
      }
      __syncwarp();
      if (q * C >= lt && (q + 1) * C <= N)
        forward(bool_tag<true>{}, slot(q), q * C, pm, d);
      else
        forward(bool_tag<false>{}, slot(q), q * C, pm, d);
    }
    const int qq = q - 1;
    if (qq >= qo0 && qq < qo1) {
      c2 x = zero2();
      const int la = min(a.halo, N - q * C);
      const E* sq = slot(q);
      const bool la_fast = q * C >= lt;
      for (int h = la - 1; h >= 0; --h) {
        k2 be = cf.be;
        if (!la_fast) {
          const int i = min(q * C + h, lt);
          be = make_k2(crow[0][i].be, crow[1][i].be);
        }
        c2 t;
        t.re = make_float2(sq[lane * PITCH + h].x, sq[(lane + 32) * PITCH + h].x);
        t.im = make_float2(sq[lane * PITCH + h].y, sq[(lane + 32) * PITCH + h].y);
        x = bwd2(be, x, t);
      }
      E* sp = slot(qq);
      if (qq * C >= lt && q * C <= N)
        backward(bool_tag<true>{}, sp, qq * C, x);
      else
        backward(bool_tag<false>{}, sp, qq * C, x);
      __syncwarp();
#pragma unroll
      for (int i = 0; i < ROWS * SPR / 32; ++i) {
        const int t = i * 32 + lane;
        const int row = t / SPR, col = t % SPR;
        const int p = qq * C + col * EP;
        const long long rr = row0 + row;
        if (rr < nrows && p < N) {
          const E* src = sp + row * PITCH + col * EP;
          if (EP == 2)
            *reinterpret_cast<float4*>(out + rr * N + p) = *reinterpret_cast<const float4*>(src);
          else
            out[rr * N + p] = *src;
        }
      }
    }
    __syncwarp();
    issue(q + R - 1);
  }
  if (!TMA) cp_async_wait<0>();
}

// One row per lane, complex float, TMA in and out.  A warp owns 32
// consecutive rows; a chunk of C points of them is one 2-D TMA box of 32
// rows x 8C bytes, swizzled (64-byte rows for C = 8, 128-byte rows for
// C = 16: 16-byte unit u of row r lands at unit u ^ s(r)), so that each lane
// reads and writes its own row with conflict-free 16-byte accesses.  The
// lane advances its points by H1 (with the pending scale), solves the chunk
// in the unfolded form of k_sweep_s1t (d_p = m2 psi_p + al d_{p-1};
// z_p = d_p + be z_{p+1}; psi'_p = z_p - psi_p, psi after H1), keeps the
// H1-advanced points in the slot for the back substitution one chunk later,
// overwrites them with the results, and the slot leaves as one TMA box
// store.  Ring of R + 1 slots as in k_sweep_s1t.  C = 16 runs 8 warps per
// SM with all the registers it wants (166); capped at 144 so that 14 warps
// fit (one wave of units on the 512 x 512 x 128 state) it measured slower
// on GB300 (141 against 114 us per sweep).
template <int C, bool IMAG, int RING>
__global__ void __launch_bounds__(C == 8 ? 512 : 256) k_sweep_x1t(const __grid_constant__ CUtensorMap map,
                                                   const __grid_constant__ CUtensorMap omap,
                                                   const stream_args a) {
  constexpr int NS = RING + 1;        // slots per warp
  constexpr int ROWS = 32;
  constexpr int U = C / 2;            // 16-byte units per row
  constexpr int SLOT = ROWS * C;      // float2 per slot (2 or 4 KB)
  static_assert((C == 8 || C == 16) && (SLOT * 8) % 1024 == 0 && NS <= 8, "TMA slots");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[16 * 8];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  if (a.ring != RING || blockDim.x > (C == 8 ? 512u : 256u) ||
      dynamic_smem_bytes() < (blockDim.x >> 5) * (unsigned)(NS * SLOT * 8) + 1024u) {
    if (threadIdx.x == 0) atomicOr(a.flags, 2);
    return;
  }
  // swizzled boxes repeat every 1024 bytes of shared address: align to it
  unsigned char* sbase = smem_raw + ((1024 - (smem_addr(smem_raw) & 1023)) & 1023);
  float2* ring = reinterpret_cast<float2*>(sbase) + (size_t)wib * NS * SLOT;
  uint64_t* bar = bars + wib * 8;
  const long long nrows = a.nlines;
  const long long ngroups = (nrows + ROWS - 1) / ROWS;
  if (lane == 0) {
    for (int i = 0; i < NS; ++i) mbar_init(&bar[i], 1);
    mbar_fence_init();
  }
  __syncwarp();
  // launched programmatically: the next sweep's blocks may be scheduled as
  // SMs free up; the previous kernel's state and pending scale are complete
  // and visible past this wait, and nothing above touched global memory
  griddep_launch_dependents();
  griddep_wait();
  const uint64_t pol_last = l2_evict_last();
  unsigned ph = 0;  // phase parity of every slot's barrier, kept from unit to unit
  bool good = true;
  // units (32 rows and one segment of them) in a fixed round-robin order
  // over the resident warps
  const long long nunits = ngroups * a.nseg;
  const long long wstride = (long long)gridDim.x * (blockDim.x >> 5);
  for (long long wg = (long long)blockIdx.x * (blockDim.x >> 5) + wib; wg < nunits && good;
       wg += wstride) {
    const long long g = wg % ngroups;
    const int sg = (int)(wg / ngroups);
    const long long row0 = g * ROWS;
    const long long row = row0 + lane;
    const bool act = row < nrows;
    const int N = a.len, nch = (N + C - 1) / C, lt = a.lt;
    const int qo0 = sg * a.seg_chunks, qo1 = min(nch, qo0 + a.seg_chunks);
    const int qa = max(0, qo0 - a.warm), qb = min(nch, qo1 + 1);
    const int jj = act ? (int)(row % a.ny) : 0, kk = act ? (int)(row / a.ny) : 0;
    const int li = jj;  // the line's coefficient line
    const float2* tab = a.coefT;
    const int tl = a.tlines;
    float2 M2R, M2I, ALR, ALI, BER, BEI;
    wsplit(coef_plane(tab, tl, lt, 0, lt, li, pol_last), M2R, M2I);
    wsplit(coef_plane(tab, tl, lt, 1, lt, li, pol_last), ALR, ALI);
    wsplit(coef_plane(tab, tl, lt, 2, lt, li, pol_last), BER, BEI);
    const float2 NEG1 = make_float2(-1.f, -1.f);
    const float yv = (float)(a.y0 + (double)jj * a.hy), zv = (float)(a.z0 + (double)kk * a.hz);
    const float vyz = (float)a.hnu2 * yv * yv + (float)a.hlam2 * zv * zv;
    const float sc = (float)(*a.scale), hg2 = (float)a.hgam2, dt = (float)a.dt, gg = (float)a.g;
    const float xs = (float)a.x0, hx = (float)a.hx;
    const float2 SC = make_float2(sc, sc);
    auto h1 = [&](float2 v, int p) -> float2 {
      v = __fmul2_rn(SC, v);
      const float x = fmaf((float)p, hx, xs);
      const float en = fmaf(gg, fmaf(v.x, v.x, v.y * v.y), fmaf(hg2 * x, x, vyz));
      if (IMAG) {
        const float f = __expf(-dt * en);
        return __fmul2_rn(make_float2(f, f), v);
      } else {
        float c1, s1;
        rot_t(dt * en, &c1, &s1);
        return rotate_f(v, c1, s1);
      }
    };
    // imaginary time: the factor sc exp(-dt (V + g sc^2 |v|^2)) of a raw
    // point v as one base-2 exponential of a quadratic in x and |v|^2, the
    // pending scale folded in as log2(sc)
    const float L2E = 1.4426950408889634f;
    const float k1 = -dt * gg * sc * sc * L2E, kx = -dt * hg2 * L2E;
    const float k0 = fmaf(-dt * L2E, vyz, log2f(sc));
    auto h1i = [&](float2 v, float x) -> float2 {
      const float t = fmaf(k1, fmaf(v.x, v.x, v.y * v.y), fmaf(kx * x, x, k0));
      float f;
      asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(f) : "f"(t));
      return __fmul2_rn(make_float2(f, f), v);
    };
    auto fwd = [](float2 mr, float2 mi, float2 lr, float2 li, float2 psi, float2 d) -> float2 {
      float2 A = __fmul2_rn(mr, psi), B = __fmul2_rn(mi, psi);
      A = __ffma2_rn(lr, d, A);
      B = __ffma2_rn(li, d, B);
      return make_float2(A.x - B.y, A.y + B.x);
    };
    auto bstep = [](float2 br, float2 bi, float2 z, float2 dp) -> float2 {
      const float2 A = __ffma2_rn(br, z, dp), B = __fmul2_rn(bi, z);
      return make_float2(A.x - B.y, A.y + B.x);
    };
    const int swz = C == 8 ? (lane >> 1) & 3 : lane & 7;  // this row's unit swizzle
    auto unit = [&](int sl, int u) -> float4* {
      return reinterpret_cast<float4*>(ring + (size_t)sl * SLOT + lane * C) + (u ^ swz);
    };
    // the row pieces of a box (64 or 128 bytes of each of 32 rows) are loaded
    // with the normal L2 policy: with evict_first the rest of the lines they
    // share with the next chunk left L2 before that chunk's load, and on a
    // state larger than L2 the sweep read 14-43% of the state twice from DRAM
    auto issue = [&](int q, int sl) {  // lane 0
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(&bar[sl], (unsigned)(SLOT * 8));
      tma_load_2d(ring + (size_t)sl * SLOT, &map, 2 * q * C, (int)row0, &bar[sl]);
    };
    if (lane == 0) {
      bulk_wait_read<0>();  // the previous unit's stores have left their slots
      for (int q = qa; q < min(qa + RING - 1, qb); ++q) issue(q, q - qa);
    }
    __syncwarp();
    float2 d = make_float2(0.f, 0.f);
    int sq = 0;  // slot of chunk q
    // forward over chunk q into cur[], back substitution and store of chunk
    // q - 1 from prv[], then the load of chunk q + R - 1 (into chunk q - 2's slot)
    auto step = [&](int q, float2 (&cur)[C], float2 (&prv)[C]) -> bool {
      const int sp = sq == 0 ? NS - 1 : sq - 1;
      if (q < qb) {
        if (!__all_sync(0xffffffffu, mbar_wait(&bar[sq], (ph >> sq) & 1u))) {
          int s = sq;
          for (int r = q + 1; r < min(q + RING - 1, qb); ++r) {
            s = s + 1 == NS ? 0 : s + 1;
            mbar_wait(&bar[s], (ph >> s) & 1u);
          }
          if (lane == 0) atomicOr(a.flags, 4);
          return false;
        }
        ph ^= 1u << sq;
        const int p0 = q * C;
        const float xp0 = fmaf((float)p0, hx, xs);  // x of the chunk's first point
        float2 w[C];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const float4 t = *unit(sq, u);
          if (IMAG) {
            w[2 * u] = h1i(make_float2(t.x, t.y), fmaf((float)(2 * u), hx, xp0));
            w[2 * u + 1] = h1i(make_float2(t.z, t.w), fmaf((float)(2 * u + 1), hx, xp0));
          } else {
            w[2 * u] = h1(make_float2(t.x, t.y), p0 + 2 * u);
            w[2 * u + 1] = h1(make_float2(t.z, t.w), p0 + 2 * u + 1);
          }
        }
        if (p0 >= lt && p0 + C <= N) {
#pragma unroll
          for (int r = 0; r < C; ++r) {
            d = fwd(M2R, M2I, ALR, ALI, w[r], d);
            cur[r] = d;
          }
        } else {
          float2 km[C], kl[C];
          table_fwd<C>(tab, tl, lt, li, p0, pol_last, km, kl);
#pragma unroll
          for (int r = 0; r < C; ++r) {
            float2 mr, mi, lr, li;
            wsplit(km[r], mr, mi);
            wsplit(kl[r], lr, li);
            d = fwd(mr, mi, lr, li, w[r], d);
            cur[r] = d;
          }
        }
        // keep the H1-advanced points for the back substitution
#pragma unroll
        for (int u = 0; u < U; ++u)
          *unit(sq, u) = make_float4(w[2 * u].x, w[2 * u].y, w[2 * u + 1].x, w[2 * u + 1].y);
      }
      const int qq = q - 1;
      bool stored = false;
      if (qq >= qo0 && qq < qo1) {
        float2 z = make_float2(0.f, 0.f);
        if (q < qb) {
          const int p0 = q * C;
          if (p0 >= lt && p0 + C <= N) {
#pragma unroll
            for (int h = C - 1; h >= 0; --h) z = bstep(BER, BEI, z, cur[h]);
          } else {
            float2 kb[C];
            table_be<C>(tab, tl, lt, li, p0, pol_last, kb);
#pragma unroll
            for (int h = C - 1; h >= 0; --h)
              if (p0 + h < N) {
                float2 br, bi;
                wsplit(kb[h], br, bi);
                z = bstep(br, bi, z, cur[h]);
              }
          }
        }
        const int p0 = qq * C;
        if (p0 >= lt && p0 + C <= N) {
#pragma unroll
          for (int u = U - 1; u >= 0; --u) {
            const float4 t = *unit(sp, u);
            z = bstep(BER, BEI, z, prv[2 * u + 1]);
            const float2 o1 = __ffma2_rn(NEG1, make_float2(t.z, t.w), z);
            z = bstep(BER, BEI, z, prv[2 * u]);
            const float2 o0 = __ffma2_rn(NEG1, make_float2(t.x, t.y), z);
            *unit(sp, u) = make_float4(o0.x, o0.y, o1.x, o1.y);
          }
        } else {
          float2 kb[C];
          table_be<C>(tab, tl, lt, li, p0, pol_last, kb);
#pragma unroll
          for (int u = U - 1; u >= 0; --u) {
            const float4 t = *unit(sp, u);
            float2 o[2];
#pragma unroll
            for (int e = 1; e >= 0; --e) {
              const int r = 2 * u + e;
              if (p0 + r < N) {
                float2 br, bi;
                wsplit(kb[r], br, bi);
                z = bstep(br, bi, z, prv[r]);
              }
              o[e] = __ffma2_rn(NEG1, e ? make_float2(t.z, t.w) : make_float2(t.x, t.y), z);
            }
            *unit(sp, u) = make_float4(o[0].x, o[0].y, o[1].x, o[1].y);
          }
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncwarp();
        if (lane == 0) {
          tma_store_2d(&omap, 2 * qq * C, (int)row0, ring + (size_t)sp * SLOT);
          bulk_commit();
        }
        stored = true;
      }
      if (lane == 0 && q + RING - 1 < qb) {
        if (stored)
          bulk_wait_read<1>();
        else
          bulk_wait_read<0>();
        int sl = sq + NS - 2;
        if (sl >= NS) sl -= NS;
        issue(q + RING - 1, sl);
      }
      __syncwarp();
      sq = sq + 1 == NS ? 0 : sq + 1;
      return true;
    };
    float2 dA[C], dB[C];
#pragma unroll
    for (int r = 0; r < C; ++r) dA[r] = dB[r] = make_float2(0.f, 0.f);
    for (int q = qa; q <= qb; q += 2) {
      if (!step(q, dA, dB)) {
        good = false;
        break;
      }
      if (q + 1 > qb) break;
      if (!step(q + 1, dB, dA)) {
        good = false;
        break;
      }
    }
  }
  if (lane == 0) bulk_wait_all();
}

size_t x1t_smem_per_warp(int C, int R) { return (size_t)(R + 1) * 32 * C * 8; }

template <int C, int R>
static cudaError_t dispatch_x1t(bool imag, const stream_args& a, const sweep_shape& sh,
                                const void* map, const void* omap, cudaStream_t s) {
  const CUtensorMap& m = *static_cast<const CUtensorMap*>(map);
  const CUtensorMap& om = *static_cast<const CUtensorMap*>(omap);
  auto fn = imag ? k_sweep_x1t<C, true, R> : k_sweep_x1t<C, false, R>;
  cudaError_t e = allow_smem((const void*)fn);
  if (e != cudaSuccess) return e;
  const long long units = (a.nlines + 31) / 32 * a.nseg;
  int W = 1;
  unsigned blocks = 0;
  e = resident_grid((const void*)fn, units, x1t_smem_per_warp(C, R), 1024, C == 8 ? 16 : 8, &W,
                    &blocks);
  if (e != cudaSuccess) return e;
  return launch_programmatic(fn, blocks, 32 * W, x1t_smem_per_warp(C, R) * W + 1024, s, m, om, a);
}

template <int C, int R>
static cudaError_t dispatch_x2r(bool imag, bool vec16, const stream_args& a,
                                const sweep_shape& sh, const void* map, cudaStream_t s) {
  const bool tma = map != nullptr && vec16 && sh.warps_per_block <= 4;
  static const CUtensorMap none{};
  const CUtensorMap& m = tma ? *static_cast<const CUtensorMap*>(map) : none;
  auto fn = tma ? (imag ? k_sweep_x2<C, true, true, true, R> : k_sweep_x2<C, false, true, true, R>)
          : vec16 ? (imag ? k_sweep_x2<C, true, true, false, R>
                          : k_sweep_x2<C, false, true, false, R>)
                  : (imag ? k_sweep_x2<C, true, false, false, R>
                          : k_sweep_x2<C, false, false, false, R>);
  cudaError_t e = allow_smem((const void*)fn);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)sh.blocks, 32 * sh.warps_per_block, sh.smem + (tma ? 128 : 0), s>>>(m, a);
  return cudaGetLastError();
}

template <int C>
static cudaError_t dispatch_x2(bool imag, bool vec16, const stream_args& a, const sweep_shape& sh,
                               const void* map, cudaStream_t s) {
  if (sh.R == 3) return dispatch_x2r<C, 3>(imag, vec16, a, sh, map, s);
  if (sh.R == 4) return dispatch_x2r<C, 4>(imag, vec16, a, sh, map, s);
  return cudaErrorInvalidValue;
}

template <class T, int V, int C>
static cudaError_t dispatch_x(bool imag, bool vec16, const stream_args& a, const sweep_shape& sh,
                              cudaStream_t s) {
  auto fn = vec16 ? (imag ? k_sweep_x<T, V, C, true, true> : k_sweep_x<T, V, C, false, true>)
                  : (imag ? k_sweep_x<T, V, C, true, false> : k_sweep_x<T, V, C, false, false>);
  cudaError_t e = allow_smem((const void*)fn);
  if (e != cudaSuccess) return e;
  fn<<<(unsigned)sh.blocks, 32 * sh.warps_per_block, sh.smem, s>>>(a);
  return cudaGetLastError();
}

// Every (precision, V, C) combination the host can choose is instantiated
// here; anything else is rejected before a launch.
cudaError_t launch_sweep_x(bool fp64, bool imag, const stream_args& a, const sweep_shape& sh,
                           const void* map, const void* omap, cudaStream_t s) {
  if (fp64) {
    if (sh.V == 1 && sh.C == 16) return dispatch_x<double, 1, 16>(imag, true, a, sh, s);
    if (sh.V == 1 && sh.C == 64) return dispatch_x<double, 1, 64>(imag, true, a, sh, s);
    return cudaErrorInvalidValue;
  }
  if (sh.V == 2 && sh.C == 8) return dispatch_x2<8>(imag, sh.vec16, a, sh, map, s);
  if (sh.V == 2 && sh.C == 16) return dispatch_x2<16>(imag, sh.vec16, a, sh, map, s);
  // one row per lane through TMA (the host passes the swizzled 32-row maps)
  if (sh.V == 1 && (sh.C == 8 || sh.C == 16) && sh.vec16 && map && omap) {
    if (sh.C == 8) {
      if (sh.R == 3) return dispatch_x1t<8, 3>(imag, a, sh, map, omap, s);
      if (sh.R == 4) return dispatch_x1t<8, 4>(imag, a, sh, map, omap, s);
      if (sh.R == 5) return dispatch_x1t<8, 5>(imag, a, sh, map, omap, s);
      if (sh.R == 6) return dispatch_x1t<8, 6>(imag, a, sh, map, omap, s);
      return cudaErrorInvalidValue;
    }
    return sh.R == 3 ? dispatch_x1t<16, 3>(imag, a, sh, map, omap, s)
                     : dispatch_x1t<16, 4>(imag, a, sh, map, omap, s);
  }
  if (sh.V == 1 && sh.C == 16) return dispatch_x<float, 1, 16>(imag, sh.vec16, a, sh, s);
  if (sh.V == 1 && sh.C == 64) return dispatch_x<float, 1, 64>(imag, sh.vec16, a, sh, s);
  return cudaErrorInvalidValue;
}

}  // namespace rotgp
