// Stage-program builder and executors (see program.h).
#include <algorithm>
#include <cstring>

#include "../../include/fhe.h"
#include "elementwise.cuh"
#include "program.h"

using namespace fhe;

static Seg seg(const uint32_t *src, uint32_t *dst, int n, int prime, int item) {
  Seg s;
  memset(&s, 0, sizeof s);
  s.src = src;
  s.dst = dst;
  s.n = n;
  s.prime = prime;
  s.src_stride = 1;
  s.src_prime = -1;
  s.item = item;
  s.galois = 1;
  return s;
}

static void add(Stage &st, const Seg &s) {
  if (s.n > 0) st.segs.push_back(s);
}

static Stage ntt_stage(bool column, bool fwd, int pro, int epi) {
  Stage s;
  s.kind = Stage::NTT;
  s.column = column;
  s.fwd = fwd;
  s.pro = pro;
  s.epi = epi;
  return s;
}

static Stage ew_stage(int op) {
  Stage s;
  s.kind = Stage::EW;
  s.ewop = op;
  return s;
}

static Stage marker(Stage::Kind k) {
  Stage s;
  s.kind = k;
  return s;
}

// the two passes of one transform: one single-pass cluster stage when the context asks for
// it and the kernel exists for the pair's prologue and epilogue, else two stages
static void push_transform(fhe_ctx *c, Program &P, const Stage &first, const Stage &second) {
  if ((c->tabs.ntt_single || c->tabs.ntt_persist) && fhe::ntt_single_pass_ok(c->tabs, first.pro, second.epi, first.fwd)) {
    Stage f = first;
    f.kind = Stage::NTT1;
    f.epi = second.epi;
    f.segs2 = second.segs;
    P.stages.push_back(f);
    return;
  }
  P.stages.push_back(first);
  P.stages.push_back(second);
}

int build_program(fhe_ctx *c, const std::vector<Item> &items, bool fused, Program &P) {
  const size_t N = c->N;
  const int L = c->L, K = c->K, A = c->alpha;
  P.ks.clear();
  P.stages.clear();
  int max_slot = 0;
  for (const Item &it : items) max_slot = std::max(max_slot, std::max(it.slot, it.ext_slot));
  int rc = ensure_slots(c, max_slot + 1);
  if (rc != FHE_OK) return rc;

  // per-item arguments and the polynomial each item key-switches
  std::vector<const uint32_t *> dpoly(items.size(), nullptr);
  for (size_t i = 0; i < items.size(); i++) {
    const Item &it = items[i];
    const fhe_ctx::Slot &S = c->slots[it.slot];
    const size_t poly = (size_t)it.level * N;
    KsArgs k;
    memset(&k, 0, sizeof k);
    k.ext = S.EXT;
    k.key = it.key;
    k.pinv = c->d_pinv;
    k.pmod = c->d_pmod;
    k.level = it.level;
    k.n_ext = it.level + K;
    k.beta = c->beta(it.level);
    k.alpha = A;
    k.L = L;
    k.K = K;
    k.galois_own = k.galois_ext = k.galois_add = 1;
    switch (it.kind) {
      case IT_KS:
        dpoly[i] = it.in;
        break;
      case IT_ROTATE:
        dpoly[i] = it.in + poly;
        k.galois_own = k.galois_add = it.galois;
        k.addp = it.in;
        break;
      case IT_RELIN:
        dpoly[i] = S.D + 2 * poly;
        k.addp = S.D;
        k.add_c1 = 1;
        break;
      case IT_MODUP:  // `in` is the polynomial itself
        dpoly[i] = it.in;
        break;
      case IT_MODDOWN:
        k.ext = c->slots[it.ext_slot].EXT;
        k.galois_own = k.galois_ext = k.galois_add = it.galois;
        k.addp = it.in;
        break;
      case IT_IPX:
        k.ext = c->slots[it.ext_slot].EXT;
        k.galois_own = k.galois_ext = k.galois_add = it.galois;
        k.addp = it.in2;
        break;
      case IT_MDX:
        break;
    }
    k.own = it.kind == IT_MODDOWN ? it.in + poly : it.kind == IT_IPX ? it.in : dpoly[i];
    // the plain pipeline gathers the rotated polynomial into TMP first
    if (!fused && it.kind == IT_ROTATE && it.galois != 1u) {
      k.own = S.TMP;
      k.galois_own = 1;
    }
    P.ks.push_back(k);
  }
  auto has_modup = [](const Item &it) { return it.kind != IT_MODDOWN && it.kind != IT_IPX && it.kind != IT_MDX; };
  auto has_ip = [](const Item &it) { return it.kind != IT_MODUP && it.kind != IT_MDX; };
  auto has_moddown = [](const Item &it) { return it.kind != IT_MODUP && it.kind != IT_IPX; };

  // ---- HMult tensor
  Stage tensor = ew_stage(EW_TENSOR);
  for (size_t i = 0; i < items.size(); i++)
    if (items[i].kind == IT_RELIN) {
      Seg s = seg(items[i].in, c->slots[items[i].slot].D, items[i].level, 0, (int)i);
      s.src2 = items[i].in2;
      add(tensor, s);
    }
  if (!tensor.segs.empty()) P.stages.push_back(tensor);

  // ---- stage 1: ModUp
  bool any_rot = false;
  for (const Item &it : items) any_rot |= has_modup(it) && it.kind == IT_ROTATE && it.galois != 1u;
  Stage gather = ew_stage(EW_GATHER);
  Stage i1 = ntt_stage(false, false, (fused && any_rot) ? PRO_GATHER : PRO_PLAIN, EPI_LAZY);
  Stage i2 = ntt_stage(true, false, PRO_PLAIN, EPI_SCALE);
  Stage sc = ew_stage(EW_SCALE);
  Stage bc;
  bc.kind = Stage::BCONV;
  Stage n1 = ntt_stage(true, true, PRO_PLAIN, EPI_LAZY);
  for (size_t i = 0; i < items.size(); i++) {
    const Item &it = items[i];
    if (!has_modup(it)) continue;
    const fhe_ctx::Slot &S = c->slots[it.slot];
    const int level = it.level, n_ext = level + K, beta = c->beta(level);
    const uint32_t *src = dpoly[i];
    if (!fused && it.kind == IT_ROTATE && it.galois != 1u) {
      Seg gs = seg(src, S.TMP, level, 0, (int)i);
      gs.galois = it.galois;
      add(gather, gs);
      src = S.TMP;
    }
    add(i1, seg(src, S.Y, level, 0, (int)i));
    Seg y = seg(S.Y, S.Y, level, 0, (int)i);
    if (fused) y.scale = c->d_mu_scale + (size_t)(level - 1) * L;
    add(i2, y);
    Seg z = seg(S.Y, S.Y, level, 0, (int)i);
    z.scale = c->d_mu_qhinv + (size_t)(level - 1) * L;
    add(sc, z);
    for (int j = 0; j < beta; j++) {
      const int lo = j * A, hi = std::min((j + 1) * A, level);
      BconvGroup g;
      memset(&g, 0, sizeof g);
      g.in = S.Y + (size_t)lo * N;
      g.out = S.EXT + (size_t)j * n_ext * N;
      g.T = c->modup_T[(size_t)(level - 1) * c->dnum + j];
      g.omap = c->modup_map[(size_t)(level - 1) * c->dnum + j];
      g.n_in = hi - lo;
      g.n_out = n_ext - (hi - lo);
      g.Btc = c->modup_Btc[(size_t)(level - 1) * c->dnum + j];
      g.npad = tc_npad(g.n_out);
      bc.groups.push_back(g);
      bc.max_in = std::max(bc.max_in, g.n_in);
      bc.max_out = std::max(bc.max_out, g.n_out);
      uint32_t *e = S.EXT + (size_t)j * n_ext * N;
      add(n1, seg(e, e, lo, 0, (int)i));
      add(n1, seg(e + (size_t)hi * N, e + (size_t)hi * N, level - hi, hi, (int)i));
      add(n1, seg(e + (size_t)level * N, e + (size_t)level * N, K, L, (int)i));
    }
  }
  if (!i1.segs.empty()) {
    if (!fused && !gather.segs.empty()) P.stages.push_back(gather);
    push_transform(c, P, i1, i2);
    if (!fused) P.stages.push_back(sc);
    P.stages.push_back(bc);
    Stage n2 = n1;
    n2.column = false;
    n2.epi = EPI_PLAIN;
    push_transform(c, P, n1, n2);
  }

  // ---- stages 2 and 3: inner product, ModDown
  Stage ipq;
  ipq.kind = Stage::IP;
  Stage ipp = ipq;
  Stage ipn;  // fused special-limb inner product + first inverse pass (items with plain digits)
  ipn.kind = Stage::IPN;
  Stage m1 = ntt_stage(false, false, PRO_PLAIN, EPI_LAZY);
  Stage m2 = ntt_stage(true, false, PRO_PLAIN, EPI_SCALE);
  Stage msc = ew_stage(EW_SCALE);
  Stage mbc;
  mbc.kind = Stage::BCONV;
  Stage r1 = ntt_stage(true, true, PRO_PLAIN, EPI_LAZY);
  Stage r2 = ntt_stage(false, true, PRO_PLAIN, fused ? EPI_COMBINE : EPI_PLAIN);
  Stage cb = ew_stage(EW_COMBINE);
  for (size_t i = 0; i < items.size(); i++) {
    const Item &it = items[i];
    const fhe_ctx::Slot &S = c->slots[it.slot];
    const int level = it.level, n_ext = level + K;
    const KsArgs &k = P.ks[i];
    // u: the slot's workspace, the caller's extended-basis output (IPX) or input (MDX)
    uint32_t *U = it.kind == IT_IPX ? it.out : it.kind == IT_MDX ? const_cast<uint32_t *>(it.in) : S.U;
    // the fused kernel takes the special limbs of a key switch whose digits are read directly
    const bool fuse = fused && c->fuse_ip_md && c->logn == 16 && has_ip(it) && has_moddown(it) &&
                      k.galois_ext == 1u && c->beta(level) <= 4;
    if (fuse) {
      Seg f = seg(nullptr, S.UC, K, L, (int)i);
      f.t0 = level;
      f.key_row0 = L;
      add(ipn, f);
    }
    if (has_ip(it)) {
      ipq.gather_own |= k.galois_own != 1u;
      ipq.gather_ext |= k.galois_ext != 1u;
      ipq.add_c1 |= k.addp && k.add_c1;
      Seg a = seg(nullptr, U, level, 0, (int)i);
      a.t0 = 0;
      a.key_row0 = 0;
      add(ipq, a);
      if (!fuse) {
        Seg b = seg(nullptr, U + (size_t)level * N, K, L, (int)i);
        b.t0 = level;
        b.key_row0 = L;
        add(ipp, b);
      }
    }
    if (!has_moddown(it)) continue;
    const int npoly = it.kind == IT_MDX ? it.npoly : 2;
    for (int cc = 0; cc < npoly; cc++) {
      uint32_t *uc = S.UC + (size_t)cc * K * N, *r = S.R + (size_t)cc * level * N;
      if (!fuse) add(m1, seg(U + ((size_t)cc * n_ext + level) * N, uc, K, L, (int)i));
      Seg x = seg(uc, uc, K, L, (int)i);
      if (fused) x.scale = c->d_md_scale;
      add(m2, x);
      Seg y = seg(uc, uc, K, L, (int)i);
      y.scale = c->d_md_phinv;
      add(msc, y);
      BconvGroup g;
      memset(&g, 0, sizeof g);
      g.in = uc;
      g.out = r;
      g.T = c->d_mdT;
      g.omap = c->d_mdmap;
      g.n_in = K;
      g.n_out = level;
      g.Btc = c->d_md_Btc;
      g.npad = tc_npad(level);
      mbc.groups.push_back(g);
      mbc.max_in = std::max(mbc.max_in, K);
      mbc.max_out = std::max(mbc.max_out, level);
      add(r1, seg(r, r, level, 0, (int)i));
      Seg z = fused ? seg(r, it.out + (size_t)cc * level * N, level, 0, (int)i) : seg(r, r, level, 0, (int)i);
      z.src2 = U + (size_t)cc * n_ext * N;
      z.c = cc;
      add(r2, z);
      Seg w = seg(U + (size_t)cc * n_ext * N, it.out + (size_t)cc * level * N, level, 0, (int)i);
      w.src2 = r;
      w.c = cc;
      add(cb, w);
    }
  }
  ipp.gather_own = ipq.gather_own;
  ipp.gather_ext = ipq.gather_ext;
  ipp.add_c1 = ipq.add_c1;
  // complementary pipelining (Section IV-B): the q-limb inner product on an auxiliary
  // branch beside ModDown's special-limb chain; otherwise one launch over all limbs
  const bool has_md = !m2.segs.empty();
  const bool split = fused && c->comp_pipe && has_md && !ipq.segs.empty();
  if (!ipq.segs.empty()) {
    if (split) {
      P.stages.push_back(marker(Stage::FORK));
      ipq.aux = true;
      P.stages.push_back(ipq);
      P.stages.push_back(marker(Stage::JOIN_RECORD));
      if (!ipp.segs.empty()) P.stages.push_back(ipp);
    } else {
      Stage all = ipq;
      all.segs.insert(all.segs.end(), ipp.segs.begin(), ipp.segs.end());
      P.stages.push_back(all);
    }
  }
  if (has_md) {
    if (!ipn.segs.empty()) {
      // the fused stage replaces the first inverse pass of its items: the other items' first
      // pass, then one column pass over every item's special limbs
      P.stages.push_back(ipn);
      if (!m1.segs.empty()) P.stages.push_back(m1);
      P.stages.push_back(m2);
    } else {
      push_transform(c, P, m1, m2);
    }
    if (!fused) P.stages.push_back(msc);
    P.stages.push_back(mbc);
    if ((c->tabs.ntt_single || c->tabs.ntt_persist) && fhe::ntt_single_pass_ok(c->tabs, r1.pro, r2.epi, true)) {
      // the single-pass transform reads u's q-limbs in its epilogue: join before it
      if (split) P.stages.push_back(marker(Stage::JOIN_WAIT));
      push_transform(c, P, r1, r2);
    } else {
      P.stages.push_back(r1);
      if (split) P.stages.push_back(marker(Stage::JOIN_WAIT));
      P.stages.push_back(r2);
    }
    if (!fused) P.stages.push_back(cb);
  }
  return FHE_OK;
}

// ------------------------------------------------------------------ execution

static cudaError_t launch_stage(fhe_ctx *c, const Stage &st, const SegList &sl, const BconvArgs &ba,
                                cudaStream_t s, int lane, const SegList *sl2) {
  cudaStream_t aux = lane > 0 ? c->lanes[lane].aux : c->aux;
  cudaEvent_t ev_fork = lane > 0 ? c->lanes[lane].fork : c->ev_fork;
  cudaEvent_t ev_join = lane > 0 ? c->lanes[lane].join : c->ev_join;
  // while tracing, the auxiliary branch runs on the main stream, so that every
  // kernel's event interval holds that kernel alone
  const bool serial = c->tabs.tracer != nullptr;
  cudaStream_t q = st.aux && !serial ? aux : s;
  if (serial && (st.kind == Stage::FORK || st.kind == Stage::JOIN_RECORD || st.kind == Stage::JOIN_WAIT))
    return cudaSuccess;
  switch (st.kind) {
    case Stage::NTT: return launch_ntt_pass(c->tabs, st.column, st.fwd, st.pro, st.epi, sl, q);
    case Stage::NTT1: return launch_ntt_single(c->tabs, st.fwd, st.pro, st.epi, sl, *sl2, q);
    case Stage::EW: return launch_ew(c->tabs, st.ewop, sl, q);
    case Stage::IP: return launch_ip(c->tabs, sl, st.gather_own, st.gather_ext, st.add_c1, c->dnum, q);
    case Stage::IPN: return launch_ip_intt(c->tabs, sl, std::min(c->dnum, 4), q);
    case Stage::BCONV:
      return c->bconv_mode == FHE_BCONV_TC ? launch_bconv_tc(c->tabs, ba, st.max_in, st.max_out, q, c->tabs.tc_k)
                                           : launch_bconv(c->tabs, ba, st.max_in, st.max_out, q);
    case Stage::FORK: {
      cudaError_t e = cudaEventRecord(ev_fork, s);
      return e != cudaSuccess ? e : cudaStreamWaitEvent(aux, ev_fork, 0);
    }
    case Stage::JOIN_RECORD: return cudaEventRecord(ev_join, aux);
    case Stage::JOIN_WAIT: return cudaStreamWaitEvent(s, ev_join, 0);
  }
  return cudaErrorInvalidValue;
}

bool program_fits_inline(const Program &P) {
  if ((int)P.ks.size() > kMaxInlineItems) return false;
  for (const Stage &st : P.stages)
    if ((int)st.segs.size() > kMaxSeg || (int)st.groups.size() > kMaxBconvGroups) return false;
  return true;
}

int run_program_inline(fhe_ctx *c, const Program &P, cudaStream_t s) {
  if (!program_fits_inline(P)) return fhe_fail(FHE_EINVAL, "internal: program does not fit inline launch arguments");
  SegList sl, sl2;
  BconvArgs ba;
  for (const Stage &st : P.stages) {
    memset(&sl, 0, sizeof sl);
    memset(&sl2, 0, sizeof sl2);
    memset(&ba, 0, sizeof ba);
    for (const Seg &x : st.segs) {
      sl.seg[sl.nseg++] = x;
      sl.total += x.n;
    }
    for (const Seg &x : st.segs2) {
      sl2.seg[sl2.nseg++] = x;
      sl2.total += x.n;
    }
    for (size_t i = 0; i < P.ks.size(); i++) sl.ks[i] = sl2.ks[i] = P.ks[i];
    if (st.kind == Stage::IP && st.gather_ext) {
      // the hoisted inner product takes the limbs limb by limb across runs of like segments
      // (the rotations of a hoisted set, which read the same digit limbs), at most four runs
      int g = 0;
      bool ok = true;
      for (int i = 0; i < sl.nseg && ok; i++) {
        const bool same = i > 0 && sl.seg[i].n == sl.seg[i - 1].n && sl.seg[i].t0 == sl.seg[i - 1].t0;
        if (same) {
          sl.lm_count[g - 1]++;
        } else if (g < 4) {
          sl.lm_first[g] = i;
          sl.lm_count[g++] = 1;
        } else {
          ok = false;
        }
      }
      sl.lm_groups = ok ? g : 0;
    }
    for (const BconvGroup &g : st.groups) ba.g[ba.ngroups++] = g;
    ba.lazy = 1;  // every conversion of a program feeds a forward NTT
    cudaError_t e = launch_stage(c, st, sl, ba, s, 0, &sl2);
    if (e != cudaSuccess) return fhe_fail(FHE_ECUDA, "stage launch: %s", cudaGetErrorString(e));
  }
  return FHE_OK;
}

int upload_program(fhe_ctx *c, const Program &P, DevProgram &D) {
  // one device buffer: per-item arguments, then per stage its segments, limb map and groups
  size_t bytes = sizeof(KsArgs) * P.ks.size();
  auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
  bytes = align(bytes);
  std::vector<size_t> seg_off(P.stages.size()), map_off(P.stages.size()), grp_off(P.stages.size());
  std::vector<size_t> seg2_off(P.stages.size()), map2_off(P.stages.size());
  for (size_t i = 0; i < P.stages.size(); i++) {
    const Stage &st = P.stages[i];
    int total = 0, total2 = 0;
    for (const Seg &x : st.segs) total += x.n;
    for (const Seg &x : st.segs2) total2 += x.n;
    seg_off[i] = bytes;
    bytes = align(bytes + sizeof(Seg) * st.segs.size());
    map_off[i] = bytes;
    bytes = align(bytes + sizeof(int2) * total);
    grp_off[i] = bytes;
    bytes = align(bytes + sizeof(BconvGroup) * st.groups.size());
    seg2_off[i] = bytes;
    bytes = align(bytes + sizeof(Seg) * st.segs2.size());
    map2_off[i] = bytes;
    bytes = align(bytes + sizeof(int2) * total2);
  }
  std::vector<char> host(bytes, 0);
  memcpy(host.data(), P.ks.data(), sizeof(KsArgs) * P.ks.size());
  for (size_t i = 0; i < P.stages.size(); i++) {
    const Stage &st = P.stages[i];
    memcpy(host.data() + seg_off[i], st.segs.data(), sizeof(Seg) * st.segs.size());
    // limb map: transform stages list their limbs grouped by prime (stable), so that the
    // streaming passes' consecutive units share twiddles; the order of limbs within a launch
    // does not change any result, and NTT1's two lists get the same permutation (same
    // segment sizes and primes)
    const bool by_prime = st.kind == Stage::NTT || st.kind == Stage::NTT1;
    auto fill_map = [by_prime](const std::vector<Seg> &segs, int2 *m) {
      std::vector<int2> v;
      for (size_t sidx = 0; sidx < segs.size(); sidx++)
        for (int w = 0; w < segs[sidx].n; w++) v.push_back(make_int2((int)sidx, w));
      if (by_prime)
        std::stable_sort(v.begin(), v.end(), [&segs](const int2 &a, const int2 &b) {
          return segs[a.x].prime + a.y < segs[b.x].prime + b.y;
        });
      std::copy(v.begin(), v.end(), m);
    };
    fill_map(st.segs, reinterpret_cast<int2 *>(host.data() + map_off[i]));
    memcpy(host.data() + grp_off[i], st.groups.data(), sizeof(BconvGroup) * st.groups.size());
    memcpy(host.data() + seg2_off[i], st.segs2.data(), sizeof(Seg) * st.segs2.size());
    fill_map(st.segs2, reinterpret_cast<int2 *>(host.data() + map2_off[i]));
  }
  if (cudaMalloc(&D.buf, bytes) != cudaSuccess) return fhe_fail(FHE_ENOMEM, "program upload: %zu bytes", bytes);
  if (cudaMemcpy(D.buf, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess)
    return fhe_fail(FHE_ECUDA, "program upload copy");
  char *base = static_cast<char *>(D.buf);
  D.lists.assign(P.stages.size(), SegList{});
  D.lists2.assign(P.stages.size(), SegList{});
  D.bargs.assign(P.stages.size(), BconvArgs{});
  for (size_t i = 0; i < P.stages.size(); i++) {
    const Stage &st = P.stages[i];
    SegList &sl = D.lists[i];
    memset(&sl, 0, sizeof sl);
    sl.nseg = (int)st.segs.size();
    for (const Seg &x : st.segs) sl.total += x.n;
    sl.dev = reinterpret_cast<const Seg *>(base + seg_off[i]);
    sl.vmap = reinterpret_cast<const int2 *>(base + map_off[i]);
    sl.ksdev = reinterpret_cast<const KsArgs *>(base);
    SegList &sl2 = D.lists2[i];
    memset(&sl2, 0, sizeof sl2);
    sl2.nseg = (int)st.segs2.size();
    for (const Seg &x : st.segs2) sl2.total += x.n;
    sl2.dev = reinterpret_cast<const Seg *>(base + seg2_off[i]);
    sl2.vmap = reinterpret_cast<const int2 *>(base + map2_off[i]);
    sl2.ksdev = reinterpret_cast<const KsArgs *>(base);
    BconvArgs &ba = D.bargs[i];
    memset(&ba, 0, sizeof ba);
    ba.ngroups = (int)st.groups.size();
    ba.lazy = 1;  // every conversion of a program feeds a forward NTT
    ba.dev = reinterpret_cast<const BconvGroup *>(base + grp_off[i]);
  }
  (void)c;
  return FHE_OK;
}

int run_program_dev(fhe_ctx *c, const Program &P, const DevProgram &D, cudaStream_t s, int lane) {
  for (size_t i = 0; i < P.stages.size(); i++) {
    cudaError_t e = launch_stage(c, P.stages[i], D.lists[i], D.bargs[i], s, lane, &D.lists2[i]);
    if (e != cudaSuccess) return fhe_fail(FHE_ECUDA, "stage launch: %s", cudaGetErrorString(e));
  }
  return FHE_OK;
}

void free_program(DevProgram &D) {
  if (D.buf) cudaFree(D.buf);
  D.buf = nullptr;
}
