// Page-table update (Sec. 4.1 "Level of Detail" and "Page Table
// Management"; evaluation "Page determination details"), run by one CTA of
// 1024 threads so that the whole update is one deterministic device step:
//
//   compact    request words != 0 -> request list, ascending page
//   LOD        d = float(0xFFFFFFFF - enc) is the page's nearest depth;
//              level = the largest l >= 1 with (f * e_l(p)) / d <= tau
//              (screen-space error in pixels), else 0
//   stage 1    entries holding a requested page at the requested level mark
//              it required and record the frame; entries with nothing
//              required are free
//   stage 2    unmatched requests ordered by (seen directly first, nearest
//              first, page id); the longest prefix whose level-page bytes
//              fit the staging budget is admitted, the rest is missing;
//              per level, admitted requests first fill non-required
//              sub-slots of entries already required at that level (entry
//              order, sub-slot order), then fresh entries taken least
//              recently used first (ties: index), levels in ascending order,
//              fanout^l per entry; a fresh entry forgets what it held (the
//              few least recently used are found by a radix select, not a
//              sort of all free entries)
//   lists      copy list (priority order) with 64 KiB copy segments, missing
//              list and draw list (ascending page) with Gaussian offsets
//   fade       (LOD cross-fade, fade_frames F > 0) per requested page: a
//              running fade ages by one and ends at age F or when the page
//              needs its old level again; a page drawn last frame at another
//              level starts one from that level; stage 1 keeps the old level's
//              copy required while the fade runs (it is never copied), and
//              the draw list holds it after the page's own item, with opacity
//              weights 1 - w and w = (age + 1) / (F + 1); pages not requested
//              forget their fade
//   control    usage = drawn Gaussian capacity / pool capacity; above the
//              band tau grows by step, below it (with a level > 0 drawn) tau
//              shrinks (not below 0); step *1.01 after a same-direction move
//              within 10 frames, *0.99 after a reversal within 10 frames.
// Compiled with -fmad=false (the LOD test and the controller are fp32
// formulas evaluated exactly as written).
#include <type_traits>

#include "block_sel.cuh"
#include "renderer.cuh"

namespace vm {
namespace {

constexpr int kPer = 4;  // pages a thread takes per round of the page-indexed scans

// N exclusive block scans at once (one set of barriers)
template <int N>
struct MScan {
  int64_t warp[N][32];
};
template <int N>
__device__ void bscan_n(const int64_t *v, int64_t *pre, int64_t *total, MScan<N> &sm) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t x[N];
#pragma unroll
  for (int q = 0; q < N; ++q) {
    x[q] = v[q];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x[q], o);
      if (lane >= o) x[q] += y;
    }
    if (lane == 31) sm.warp[q][warp] = x[q];
  }
  __syncthreads();
  if (warp < N) {
    int64_t t = sm.warp[warp][lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    sm.warp[warp][lane] = t;
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < N; ++q) {
    pre[q] = (warp ? sm.warp[q][warp - 1] : 0) + x[q] - v[q];
    total[q] = sm.warp[q][31];
  }
  __syncthreads();
}

__global__ void __launch_bounds__(RT) residency_kernel(ResidencyArgs a) {
  extern __shared__ uint64_t s_keys[];
  __shared__ ScanSmem sm;
  __shared__ MScan<4> sm4;
  __shared__ int m_l[kMaxLevels], S_l[kMaxLevels];
  __shared__ int n_lvl[kMaxLevels], open_cnt[kMaxLevels], open_base[kMaxLevels], fresh_start[kMaxLevels + 1];
  __shared__ int s_nfree, s_hits;
  Ctl *ctl = a.ctl;
  const int tid = threadIdx.x;
  const int NP = a.NP, P = a.P, Smax = a.Smax, L = a.levels;
  const int frame = ctl->frame;
  const float tau = ctl->tau;
  if (tid == 0) s_hits = 0;
  if (tid < kMaxLevels) {
    int m = a.page_size, S = 1;
    for (int l = 0; l < tid; ++l) { m /= a.fanout; S *= a.fanout; }
    m_l[tid] = m;
    S_l[tid] = S;
  }
  __syncthreads();

  // ---- 1. request list; per-page scratch reset (kPer consecutive pages a
  // thread, one block scan a round)
  int64_t nreq = 0, ndir = 0, tot;
  for (int c = 0; c < NP; c += RT * kPer) {
    const int p0 = c + tid * kPer;
    uint32_t r[kPer];
    int dflag[kPer];
    int64_t v2[2] = {0, 0};
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      const int p = p0 + k;
      r[k] = p < NP ? a.req[p] : 0u;
      dflag[k] = (p < NP && r[k] != 0u) ? (int)a.direct[p] : 0;
      if (p < NP) {
        a.reqlev[p] = -1;
        a.matched[p] = 0;
        a.draw_info[p] = -1;
        if (a.fade_frames > 0) { a.fade_lev[p] = -1; a.fade_info[p] = -1; }
      }
      v2[0] += r[k] != 0u;
      v2[1] += dflag[k];
    }
    int64_t pre2[2], tot2[2];
    bscan_n<2>(v2, pre2, tot2, *reinterpret_cast<MScan<2> *>(&sm4));
    int64_t o = nreq + pre2[0];
#pragma unroll
    for (int k = 0; k < kPer; ++k)
      if (r[k] != 0u) a.requests[o++] = make_int4(p0 + k, (int)r[k], dflag[k], 0);
    nreq += tot2[0];
    ndir += tot2[1];
  }
  __syncthreads();
  // ---- 2. LOD choice
  for (int i = tid; i < nreq; i += RT) {
    const int4 q = a.requests[i];
    int lev = 0;
    if (a.lod_on && L > 1) {
      const float d = __uint_as_float(0xFFFFFFFFu - (uint32_t)q.y);
      for (int l = L - 1; l >= 1; --l) {
        const float sse = (a.f_px * a.err[(int64_t)q.x * L + l]) / d;
        if (sse <= tau) { lev = l; break; }
      }
    }
    a.requests[i].w = lev;
    a.reqlev[q.x] = lev;
  }
  __syncthreads();
  // ---- 2b. cross-fade state of the requested pages (state word: cur + 1 |
  // (from + 1) << 8 | age << 16, valid only when stamped with the previous
  // frame: a page not requested last frame starts from nothing)
  const int F = a.fade_frames;
  if (F > 0) {
    for (int i = tid; i < nreq; i += RT) {
      const int p = a.requests[i].x;
      const int l = a.requests[i].w;
      const int32_t w = a.fade_frame[p] == frame - 1 ? a.fade_state[p] : 0;
      a.fade_frame[p] = frame;
      const int cur = (w & 0xFF) - 1;
      int frm = ((w >> 8) & 0xFF) - 1, age = (w >> 16) & 0xFFFF;
      if (frm >= 0) {
        ++age;
        if (age >= F || frm == l) frm = -1;
      }
      if (cur >= 0 && l != cur) {
        frm = cur;
        age = 0;
      }
      if (frm < 0) age = 0;
      a.fade_state[p] = (cur + 1) | ((frm + 1) << 8) | (age << 16);
      a.fade_lev[p] = frm;
    }
    __syncthreads();
  }
  // ---- 3. stage 1 (a copy of the loop without the fade's test when it is off)
  auto stage1 = [&](auto fade_on) {
    constexpr bool FADE = decltype(fade_on)::value;
    for (int e = tid; e < P; e += RT) {
      const int l = a.pt_lod[e];
      int any = 0;
      if (l >= 0) {
        for (int s = 0; s < S_l[l]; ++s) {
          const int64_t k = (int64_t)e * Smax + s;
          const int p = a.pt_slot[k];
          const int r = (p >= 0 && a.reqlev[p] == l) ? 1 : 0;
          // the old level of a running cross-fade, when resident, stays required
          const int rf = (FADE && !r && p >= 0 && a.fade_lev[p] == l) ? 1 : 0;
          a.required[k] = (uint8_t)(r | rf);
          if (r) {
            a.matched[p] = 1;
            a.draw_info[p] = (int)k;
            any = 1;
            if (a.pf_flag[k]) { atomicAdd(&s_hits, 1); a.pf_flag[k] = 0; }
          }
          if (FADE && rf) {
            a.fade_info[p] = (int)k;
            any = 1;
          }
        }
      }
      a.any_req[e] = (uint8_t)any;
      if (any) a.pt_last[e] = frame;
    }
  };
  if (F > 0)
    stage1(std::true_type{});
  else
    stage1(std::false_type{});
  __syncthreads();
  // ---- 4. unmatched requests as priority keys
  int64_t nu = 0;
  for (int c = 0; c < nreq; c += RT) {
    const int i = c + tid;
    int4 q = make_int4(0, 0, 0, 0);
    int f = 0;
    if (i < nreq) { q = a.requests[i]; f = a.matched[q.x] ? 0 : 1; }
    const int64_t pos = bscan(f, &tot, sm);
    if (f)
      a.ukeys[nu + pos] = ((uint64_t)(q.z ? 0u : 1u) << 63) | ((uint64_t)(~(uint32_t)q.y) << 31) | (uint64_t)q.x;
    nu += tot;
  }
  __syncthreads();
  const int nu_pow = pow2_at_least((int)nu);
  const bool sort_ok = nu_pow <= a.ukey_cap;
  if (sort_ok) {
    for (int i = (int)nu + tid; i < nu_pow; i += RT) a.ukeys[i] = ~0ull;
    __syncthreads();
    bitonic(a.ukeys, nu_pow, s_keys);
  } else if (tid == 0) {
    atomicCAS(&ctl->status, 0, VM3DGS_E_CAPACITY);
  }
  __syncthreads();
  // ---- 5. admission by the staging budget (longest prefix that fits)
  int64_t nadm = 0, cum = 0;
  for (int c = 0; c < nu && sort_ok; c += RT) {
    const int i = c + tid;
    int64_t cost = 0;
    if (i < nu) {
      const int p = (int)(a.ukeys[i] & 0x7FFFFFFFull);
      cost = (int64_t)m_l[a.reqlev[p]] * a.rec;
    }
    const int64_t pre = bscan(cost, &tot, sm);
    const int ok = (i < nu && cum + pre + cost <= a.budget) ? 1 : 0;
    // admitted entries form a prefix: count them with a block reduction
    nadm += __syncthreads_count(ok);
    cum += tot;
  }
  // ---- 6. per-level rank of the admitted requests
  for (int l = 0; l < L; ++l) {
    int64_t base = 0;
    for (int c = 0; c < nadm; c += RT) {
      const int i = c + tid;
      int f = 0;
      if (i < nadm) f = a.reqlev[(int)(a.ukeys[i] & 0x7FFFFFFFull)] == l;
      const int64_t pos = bscan(f, &tot, sm);
      if (f) a.admitted_pos[i] = (int)(base + pos);
      base += tot;
    }
    if (tid == 0) n_lvl[l] = (int)base;
  }
  // ---- 7. open sub-slots: entries required this frame at level l
  int64_t obase = 0;
  for (int l = 0; l < L; ++l) {
    int64_t cnt_e = 0, cnt_s = 0;
    for (int c = 0; c < P; c += RT * kPer) {
      const int e0 = c + tid * kPer;
      int avail[kPer], elig[kPer];
      int64_t v2[2] = {0, 0};
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int e = e0 + k;
        avail[k] = 0;
        elig[k] = 0;
        if (e < P && a.any_req[e] && a.pt_lod[e] == l) {
          elig[k] = 1;
          for (int s = 0; s < S_l[l]; ++s) avail[k] += a.required[(int64_t)e * Smax + s] ? 0 : 1;
        }
        v2[0] += elig[k];
        v2[1] += avail[k];
      }
      int64_t pre2[2], tot2[2];
      bscan_n<2>(v2, pre2, tot2, *reinterpret_cast<MScan<2> *>(&sm4));
      int64_t oe = obase + cnt_e + pre2[0], os = cnt_s + pre2[1];
#pragma unroll
      for (int k = 0; k < kPer; ++k)
        if (elig[k]) {
          a.open_list[oe] = e0 + k;
          a.open_off[oe] = (int)os;
          ++oe;
          os += avail[k];
        }
      cnt_e += tot2[0];
      cnt_s += tot2[1];
    }
    if (tid == 0) { open_base[l] = (int)obase; open_cnt[l] = (int)cnt_s; }
    // sentinel count of eligible entries stored after the list
    obase += cnt_e;
    if (tid == 0) a.open_off[P + l] = (int)cnt_e;
  }
  __syncthreads();
  // ---- 8. fresh entries needed per level; free entries, least recently used first
  if (tid == 0) {
    int acc = 0;
    for (int l = 0; l < L; ++l) {
      const int rest = n_lvl[l] > open_cnt[l] ? n_lvl[l] - open_cnt[l] : 0;
      fresh_start[l] = acc;
      acc += (rest + S_l[l] - 1) / S_l[l];
    }
    fresh_start[L] = acc;
  }
  __syncthreads();
  int64_t nfree = 0;
  if (fresh_start[L] > 0) {
    for (int c = 0; c < P; c += RT * kPer) {
      const int e0 = c + tid * kPer;
      int f[kPer], nf = 0;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        f[k] = (e0 + k < P && !a.any_req[e0 + k]) ? 1 : 0;
        nf += f[k];
      }
      int64_t o = nfree + bscan(nf, &tot, sm);
#pragma unroll
      for (int k = 0; k < kPer; ++k)
        if (f[k]) a.free_keys[o++] = ((uint64_t)(uint32_t)(a.pt_last[e0 + k] + 1) << 32) | (uint32_t)(e0 + k);
      nfree += tot;
    }
    __syncthreads();
    if (fresh_start[L] < nfree && fresh_start[L] <= kSmemKeys) {
      // only the least recently used few are taken: select them
      select_smallest(a.free_keys, (int)nfree, fresh_start[L], s_keys, sm);
    } else {
      const int fp = pow2_at_least((int)nfree);
      for (int i = (int)nfree + tid; i < fp; i += RT) a.free_keys[i] = ~0ull;
      __syncthreads();
      bitonic(a.free_keys, fp, s_keys);
    }
  }
  if (tid == 0) s_nfree = (int)nfree;
  __syncthreads();
  // ---- 9. initialise the fresh entries
  {
    const int nf = fresh_start[L] < s_nfree ? fresh_start[L] : s_nfree;
    for (int64_t x = tid; x < (int64_t)nf * Smax; x += RT) {
      const int k = (int)(x / Smax), s = (int)(x % Smax);
      const int e = (int)(a.free_keys[k] & 0xFFFFFFFFull);
      a.pt_slot[(int64_t)e * Smax + s] = -1;
      a.pf_flag[(int64_t)e * Smax + s] = 0;
      if (s == 0) {
        int l = 0;
        while (l + 1 < L && fresh_start[l + 1] <= k) ++l;
        a.pt_lod[e] = l;
        a.pt_last[e] = frame;
      }
    }
  }
  __syncthreads();
  // ---- 10. placement of the admitted requests
  for (int i = tid; i < nadm; i += RT) {
    const int p = (int)(a.ukeys[i] & 0x7FFFFFFFull);
    const int l = a.reqlev[p];
    const int rho = a.admitted_pos[i];
    int64_t slot = -1;
    if (rho < open_cnt[l]) {
      const int ob = open_base[l], ne = a.open_off[P + l];
      int lo = 0, hi = ne - 1;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.open_off[ob + mid] <= rho) lo = mid; else hi = mid - 1;
      }
      const int e = a.open_list[ob + lo];
      int want = rho - a.open_off[ob + lo];
      for (int s = 0; s < S_l[l]; ++s) {
        if (a.required[(int64_t)e * Smax + s]) continue;
        if (want == 0) { slot = (int64_t)e * Smax + s; break; }
        --want;
      }
    } else {
      const int j = rho - open_cnt[l];
      const int k = fresh_start[l] + j / S_l[l];
      if (k < s_nfree) {
        const int e = (int)(a.free_keys[k] & 0xFFFFFFFFull);
        slot = (int64_t)e * Smax + j % S_l[l];
      }
    }
    if (slot >= 0) {
      a.pt_slot[slot] = p;
      a.pf_flag[slot] = 0;
      a.draw_info[p] = (int)slot;
    } else {
      a.matched[p] = 2;
    }
  }
  __syncthreads();
  // ---- 11. copy list in priority order, with copy segments
  int64_t ncopy = 0, nseg = 0, sbytes = 0;
  for (int c = 0; c < nadm; c += RT) {
    const int i = c + tid;
    int f = 0, p = 0, l = 0;
    int64_t segs = 0, bytes = 0;
    if (i < nadm) {
      p = (int)(a.ukeys[i] & 0x7FFFFFFFull);
      l = a.reqlev[p];
      f = a.matched[p] != 2;
      bytes = f ? (int64_t)m_l[l] * a.rec : 0;
      segs = (bytes + kCopySeg - 1) / kCopySeg;
    }
    const int64_t v3[3] = {f, segs, bytes};
    int64_t pre3[3], tot3[3];
    bscan_n<3>(v3, pre3, tot3, *reinterpret_cast<MScan<3> *>(&sm4));
    if (f) {
      const int slot = a.draw_info[p];
      a.copies[ncopy + pre3[0]] = make_int4(p, l, slot / Smax, slot % Smax);
      a.copy_seg[ncopy + pre3[0]] = nseg + pre3[1];
    }
    ncopy += tot3[0];
    nseg += tot3[1];
    sbytes += tot3[2];
  }
  if (tid == 0) a.copy_seg[ncopy] = nseg;
  // non-admitted requests are missing too
  for (int i = (int)nadm + tid; i < nu; i += RT) a.matched[(int)(a.ukeys[i] & 0x7FFFFFFFull)] = 2;
  __syncthreads();
  // ---- 12. missing list and draw list, ascending page (a fading page: its
  // own item, then its old level's); draw offsets and weights.  Counts are
  // scanned two to a word (missing | items << 32, levels > 0 | fading << 32:
  // each below 2^31)
  int64_t nmiss = 0, ndraw = 0, gsum = 0, nlod = 0, nfade = 0;
  auto step12 = [&](auto fade_on) {
    constexpr bool FADE = decltype(fade_on)::value;
    for (int c = 0; c < NP; c += RT * kPer) {
      const int p0 = c + tid * kPer;
      int fm[kPer], fd[kPer], ff[kPer];
      int64_t v3[3] = {0, 0, 0};
  #pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int p = p0 + k;
        fm[k] = 0; fd[k] = 0; ff[k] = 0;
        if (p < NP) {
          fm[k] = a.matched[p] == 2;
          fd[k] = a.draw_info[p] >= 0 && !fm[k];
          ff[k] = FADE && a.fade_info[p] >= 0;
          if (fd[k]) {
            const int lv = a.reqlev[p];
            v3[1] += m_l[lv];
            v3[2] += lv > 0;
          }
          if (FADE && ff[k]) {
            const int lv = a.fade_lev[p];
            v3[1] += m_l[lv];
            v3[2] += lv > 0;
          }
        }
        v3[0] += (int64_t)fm[k] | ((int64_t)(fd[k] + ff[k]) << 32);
        v3[2] += (int64_t)(fd[k] & ff[k]) << 32;
      }
      int64_t pre3[3], tot3[3];
      bscan_n<3>(v3, pre3, tot3, *reinterpret_cast<MScan<3> *>(&sm4));
      int64_t om = nmiss + (pre3[0] & 0xFFFFFFFF), od = ndraw + (pre3[0] >> 32), og = gsum + pre3[1];
  #pragma unroll
      for (int k = 0; k < kPer; ++k) {
        const int p = p0 + k;
        if (fm[k]) a.missing[om++] = p;
        // weights: the new level (age + 1) / (F + 1), the old 1 - that
        float wn = 1.0f, wo = 1.0f;
        if (FADE && fd[k] && ff[k]) {
          wn = (float)(((a.fade_state[p] >> 16) & 0xFFFF) + 1) / (float)(F + 1);
          wo = 1.0f - wn;
        }
        if (fd[k]) {
          const int slot = a.draw_info[p];
          const int lv = a.reqlev[p];
          a.draw[od] = make_int4(p, lv, slot / Smax, slot % Smax);
          a.draw_off[od] = og;
          a.draw_w[od] = wn;
          ++od;
          og += m_l[lv];
        }
        if (FADE && ff[k]) {
          const int slot = a.fade_info[p];
          const int lv = a.fade_lev[p];
          a.draw[od] = make_int4(p, lv, slot / Smax, slot % Smax);
          a.draw_off[od] = og;
          a.draw_w[od] = wo;
          ++od;
          og += m_l[lv];
        }
        // the level drawn this frame, for the next frame's fade
        if (FADE && p < NP && a.reqlev[p] >= 0)
          a.fade_state[p] = (a.fade_state[p] & ~0xFF) | (fd[k] ? a.reqlev[p] + 1 : 0);
      }
      nmiss += tot3[0] & 0xFFFFFFFF;
      ndraw += tot3[0] >> 32;
      gsum += tot3[1];
      nlod += tot3[2] & 0xFFFFFFFF;
      nfade += tot3[2] >> 32;
    }
  };
  if (F > 0)
    step12(std::true_type{});
  else
    step12(std::false_type{});
  if (tid == 0) {
    a.draw_off[ndraw] = gsum;
    ctl->n_req = (int)nreq;
    ctl->n_direct = (int)ndir;
    ctl->n_unmatched = (int)nu;
    ctl->n_admitted = (int)nadm;
    ctl->n_copies = (int)ncopy;
    ctl->copy_segments = nseg;
    ctl->streamed_bytes = sbytes;
    ctl->n_draw = (int)ndraw;
    ctl->n_missing = (int)nmiss;
    ctl->n_resident = (int)(nreq - nu);
    ctl->n_free = s_nfree;
    ctl->n_fading = (int)nfade;
    ctl->draw_gauss = gsum;
    ctl->acc_frames += 1;
    ctl->acc_draw_gauss += gsum;
    ctl->acc_streamed_bytes += sbytes;
    ctl->acc_streamed_pages += ncopy;
    ctl->acc_missing += nmiss;
    ctl->acc_requested += nreq;
    ctl->n_hits = s_hits;
    ctl->acc_prefetch_hits += s_hits;
    const float usage = P > 0 ? (float)gsum / (float)((int64_t)P * a.page_size) : 0.0f;
    ctl->usage = usage;
    // ---- 13. LOD controller
    if (a.lod_on && L > 1) {
      const int any_lod = nlod > 0;
      int dir = 0;
      if (usage > a.usage_hi) dir = 1;
      else if (usage < a.usage_lo && any_lod) dir = -1;
      if (dir != 0) {
        const bool recent = frame - ctl->last_move <= 10;
        float step = ctl->step;
        if (recent && ctl->last_dir == dir) step = step * 1.01f;
        else if (recent && ctl->last_dir == -dir) step = step * 0.99f;
        ctl->step = step;
        float t = dir > 0 ? tau + step : tau - step;
        ctl->tau = t > 0.0f ? t : 0.0f;
        ctl->last_dir = dir;
        ctl->last_move = frame;
      }
    }
    ctl->frame = frame + 1;
  }
}

}  // namespace

void launch_residency(const ResidencyArgs &a, cudaStream_t st) {
  const int smem = kSmemKeys * (int)sizeof(uint64_t);
  max_dynamic_smem((const void *)residency_kernel, smem);
  residency_kernel<<<1, RT, smem, st>>>(a);
}

}  // namespace vm
