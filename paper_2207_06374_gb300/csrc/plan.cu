// Launch plan of one iteration over many instances (batched searches and the
// serving loop): the width-group tables of every scoring pass, the work items
// of the tensor-core screen, and the enqueue of the iteration's kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "../../include/trstmi.h"
#include "kernels.h"

namespace trstmi {

namespace {
// tile widths of the groups; kResident = whole candidate in shared memory
constexpr int kWidths[4] = {4, 2, 1, kResident};
constexpr int kNumWidths = 4;

bool is_screen_prec(int p) { return is_screen_precision(p); }

// Widest tile usable for a binary64 frame pass of this shape (<= R).
int frame64_width(int d, int N, int R) {
  while (R > 1 && (gram_smem_bytes(true, d, R) > 200 * 1024 || 16 * R >= 2 * N)) R >>= 1;
  return R;
}
}  // namespace

int BatchPlan::init(int capacity_slots, long long capacity_items, int num_sms_,
                    size_t planes_bytes_) {
  cap_slots = capacity_slots;
  cap_items = capacity_items;
  num_sms = num_sms_;
  const size_t ids_b = sizeof(int) * (size_t)cap_slots;
  const size_t beg_b = sizeof(long long) * ((size_t)cap_slots + 1);
  size_t total = 0;
  auto up = [](size_t x) { return (x + 255) / 256 * 256; };
  total += kPasses * kNumWidths * (up(ids_b) + up(beg_b));
  total += up(sizeof(ScreenSlot) * (size_t)cap_slots);
  total += up(sizeof(uint2) * (size_t)std::max<long long>(cap_items, 1));
  total += up(sizeof(unsigned long long) * kCounters);
  if (dmem.allocate(&mem, total) != cudaSuccess) { cudaGetLastError(); return TRSTMI_ENOMEM; }
  char* p = (char*)mem;
  for (int pass = 0; pass < kPasses; ++pass)
    for (int w = 0; w < kNumWidths; ++w) {
      tables[pass][w].d_ids = (int*)p; p += up(ids_b);
      tables[pass][w].d_begin = (long long*)p; p += up(beg_b);
    }
  d_screen_slots = (ScreenSlot*)p; p += up(sizeof(ScreenSlot) * (size_t)cap_slots);
  d_items = (uint2*)p; p += up(sizeof(uint2) * (size_t)std::max<long long>(cap_items, 1));
  d_counters = (unsigned long long*)p;
  planes_bytes = planes_bytes_ / 256 * 256;
  if (planes_bytes > 0 && dmem.allocate(&planes, planes_bytes) != cudaSuccess) {
    cudaGetLastError();
    planes = nullptr;
    planes_bytes = 0;
    return TRSTMI_ENOMEM;
  }
  return TRSTMI_OK;
}

void BatchPlan::destroy() {
  dmem.release(mem);
  dmem.release(planes);
  mem = nullptr;
  planes = nullptr;
  planes_bytes = 0;
}

// Whether instance sd's candidate passes run as a large instance.
bool planes_instance(const SlotDesc& sd, bool f64, bool screen, size_t planes_bytes) {
  if (f64 || sd.R == kResident || sd.N < BatchPlan::kPlanesMinN) return false;
  const size_t cands = (size_t)std::max(sd.K, screen ? sd.topk_n : 0);
  return cands * 2 * (size_t)sd.d * (size_t)sd.N * sizeof(float) <= planes_bytes;
}

int BatchPlan::rebuild(const std::vector<SlotDesc>& h, int precision_, cudaStream_t s) {
  precision = precision_;
  const int n = (int)h.size();
  if (n > cap_slots) return TRSTMI_EINVAL;
  const bool f64 = precision == TRSTMI_FP64;
  const bool screen = is_screen_prec(precision);
  maxN = 0; maxd = 0;
  for (const auto& sd : h) { maxN = std::max(maxN, sd.N); maxd = std::max(maxd, sd.d); }
  std::vector<char> is_large(n, 0);
  large.clear();
  for (int i = 0; i < n; ++i)
    if (planes && planes_instance(h[i], f64, screen, planes_bytes)) {
      is_large[i] = 1;
      large.push_back(h[i]);
    }
  ncounters = 0;
  for (int pass = 0; pass < kPasses; ++pass) {
    groups[pass].clear();
    if (!screen && pass != kPassFull) continue;
    for (int w = 0; w < kNumWidths; ++w) {
      const int R = kWidths[w];
      const bool pass64 = (pass == kPassFrame64) || (pass == kPassFull && f64);
      const bool cand_pass = pass == kPassFull || pass == kPassRescore;
      if (R == kResident && !cand_pass) continue;
      std::vector<int> ids;
      for (int i = 0; i < n; ++i) {
        // resident instances score their frames (certification passes) in
        // tiles of 16 columns
        const int r_tile = h[i].R == kResident ? 1 : h[i].R;
        const int r_i = pass == kPassFrame64 ? frame64_width(h[i].d, h[i].N, r_tile)
                        : cand_pass ? h[i].R : r_tile;
        if (r_i == R && !(cand_pass && is_large[i])) ids.push_back(i);
      }
      if (ids.empty()) continue;
      auto keff = [&](int i) {
        return pass == kPassFull ? h[i].K : pass == kPassRescore ? h[i].topk_n : 1;
      };
      // work items: one per candidate (resident) or per (candidate, tile)
      auto units = [&](int i) { return R == kResident ? 1 : tiles_at_width(h[i].N, R); };
      auto cost = [&](int i) {
        return (double)keff(i) * (R == kResident ? (double)h[i].N * h[i].N / 256.0 : units(i)) *
               h[i].d;
      };
      std::stable_sort(ids.begin(), ids.end(), [&](int x, int y) { return cost(x) > cost(y); });
      std::vector<long long> begin(ids.size() + 1, 0);
      size_t smem = 0;
      for (size_t q = 0; q < ids.size(); ++q) {
        begin[q + 1] = begin[q] + (long long)keff(ids[q]) * units(ids[q]);
        smem = std::max(smem, R == kResident ? resident_smem_bytes(pass64, h[ids[q]].d, h[ids[q]].N)
                                             : gram_smem_bytes(pass64, h[ids[q]].d, R));
      }
      Group g;
      g.R = R;
      g.f64 = pass64;
      g.d_ids = tables[pass][w].d_ids;
      g.d_begin = tables[pass][w].d_begin;
      g.count = (int)ids.size();
      g.nitems = begin.back();
      g.smem = smem;
      g.counter = ncounters++;
      int per_sm = 0;
      const cudaError_t oe = R == kResident ? batch_resident_occupancy(pass64, smem, &per_sm)
                                            : batch_score_occupancy(pass64, R, smem, &per_sm);
      if (oe != cudaSuccess || per_sm < 1) return TRSTMI_ECUDA;
      g.grid = (int)std::min<long long>(g.nitems, (long long)num_sms * per_sm);
      if (cudaMemcpyAsync(g.d_ids, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice, s) != cudaSuccess ||
          cudaMemcpyAsync(g.d_begin, begin.data(), sizeof(long long) * begin.size(),
                          cudaMemcpyHostToDevice, s) != cudaSuccess)
        return TRSTMI_ECUDA;
      groups[pass].push_back(g);
    }
  }
  // screen work items (instance, candidate), heaviest instances first
  n_items = 0;
  n_wide = 0;
  if (screen) {
    std::vector<ScreenSlot> ss(n);
    std::vector<int> order;
    for (int i = 0; i < n; ++i) {
      ss[i].phi32 = reinterpret_cast<const float2*>(h[i].phi);
      ss[i].mu2 = reinterpret_cast<unsigned int*>(h[i].mu2);
      ss[i].st = h[i].st;
      ss[i].seed = h[i].seed;
      ss[i].N = h[i].N;
      ss[i].d = h[i].d;
      if (h[i].screen) order.push_back(i);
    }
    // the instances of the d <= 32 format first, then those of the wide
    // format (32 < d <= 64), each part heaviest first
    const auto wide = [&](int i) { return screen_fmt_of(precision, h[i].d) != screen_fmt_of(precision, 1); };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
      if (wide(x) != wide(y)) return wide(y);
      const long long nx = (h[x].N + 127) / 128, ny = (h[y].N + 127) / 128;
      return nx * (nx + 1) > ny * (ny + 1);
    });
    std::vector<uint2> items;
    n_wide = 0;
    for (int i : order)
      for (int c = 0; c < h[i].K; ++c) {
        items.push_back(make_uint2((unsigned)i, (unsigned)c));
        if (wide(i)) ++n_wide;
      }
    if ((long long)items.size() > cap_items) return TRSTMI_EINVAL;
    n_items = (int)items.size();
    if (cudaMemcpyAsync(d_screen_slots, ss.data(), sizeof(ScreenSlot) * n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        (n_items && cudaMemcpyAsync(d_items, items.data(), sizeof(uint2) * items.size(),
                                    cudaMemcpyHostToDevice, s) != cudaSuccess))
      return TRSTMI_ECUDA;
  }
  return TRSTMI_OK;
}

cudaError_t BatchPlan::launch_pass(int pass, SlotDesc* d_slots, cudaStream_t s) const {
  for (const auto& g : groups[pass]) {
    cudaError_t e =
        g.R == kResident
            ? launch_batch_resident(g.f64, d_slots, g.d_ids, g.d_begin, g.count, g.nitems,
                                    d_counters + g.counter, g.smem, g.grid, s, pass)
            : launch_batch_score(g.f64, g.R, d_slots, g.d_ids, g.d_begin, g.count, g.nitems,
                                 d_counters + g.counter, g.smem, g.grid, s, pass);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

int BatchPlan::enqueue_iteration(SlotDesc* d_slots, int n, uint32_t* err, cudaStream_t s) const {
  const bool f64 = precision == TRSTMI_FP64;
  const bool screen = is_screen_prec(precision);
  if (launch_batch_begin(d_slots, n, d_counters, kCounters, f64, screen, s) != cudaSuccess)
    return TRSTMI_ECUDA;
  if (!screen) {
    if (launch_pass(kPassFull, d_slots, s) != cudaSuccess ||
        launch_large(kPassFull, s) != cudaSuccess ||
        launch_batch_decide(d_slots, n, f64, s) != cudaSuccess ||
        launch_batch_commit(d_slots, n, maxN, f64, s) != cudaSuccess)
      return TRSTMI_ECUDA;
    return TRSTMI_OK;
  }
  // rank (screen, or fp32 below the screen radius), keep the top-k, re-score
  // them in fp32, regenerate the winner in fp64 and certify it (one binary32
  // filter pass from the winner's score, binary64 pairs), decide, commit
  if (launch_screen(err, s) != cudaSuccess ||
      launch_pass(kPassFull, d_slots, s) != cudaSuccess ||
      launch_large(kPassFull, s) != cudaSuccess ||
      launch_batch_topk(d_slots, n, s) != cudaSuccess ||
      launch_pass(kPassRescore, d_slots, s) != cudaSuccess ||
      launch_large(kPassRescore, s) != cudaSuccess ||
      launch_batch_materialize64(d_slots, n, maxN, s) != cudaSuccess ||
      launch_pass(kPassFilter, d_slots, s) != cudaSuccess ||
      launch_batch_pairs64(d_slots, n, s) != cudaSuccess ||
      launch_pass(kPassFrame64, d_slots, s) != cudaSuccess ||
      launch_batch_decide_certified(d_slots, n, s) != cudaSuccess ||
      launch_batch_commit_copy(d_slots, n, maxN, maxd, s) != cudaSuccess)
    return TRSTMI_ECUDA;
  return TRSTMI_OK;
}

cudaError_t BatchPlan::launch_large(int pass, cudaStream_t s) const {
  for (const SlotDesc& sd : large) {
    const bool full = pass == kPassFull;
    // kPassFull: every candidate, while the instance ranks with the binary32
    // Gram (use_full: always in the binary32 mode); kPassRescore: the top-k
    // survivors, after the screen ranked them (use_screen)
    const uint32_t* gate = full ? &sd.st->use_full : &sd.st->use_screen;
    const int count = full ? sd.K : sd.topk_n;
    const uint32_t* cands = full ? nullptr : sd.topk;
    const float2* phi = reinterpret_cast<const float2*>(sd.phi);
    cudaError_t e = launch_gen_planes_f32(sd.N, sd.d, count, phi, sd.seed, 0u, sd.st, 0u, 0.0,
                                          reinterpret_cast<float*>(planes), s, cands, gate);
    if (e != cudaSuccess) return e;
    GramSource src{};
    src.perturb = true;
    src.phi = phi;
    src.seed = sd.seed;
    src.cand_list = cands;
    src.st = sd.st;
    src.gate = gate;
    src.planes = planes;
    e = launch_gram_f32(sd.N, sd.d, count, src,
                        full ? reinterpret_cast<unsigned int*>(sd.mu2) : sd.mu2_top, nullptr,
                        num_sms, s);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t BatchPlan::launch_screen(uint32_t* err, cudaStream_t s) const {
  const int n_narrow = n_items - n_wide;
  cudaError_t e = cudaSuccess;
  if (n_narrow > 0)
    e = launch_screen_batched(screen_fmt_of(precision, 1), d_screen_slots, d_items, n_narrow,
                              err, num_sms, s);
  if (e == cudaSuccess && n_wide > 0)
    e = launch_screen_batched(screen_fmt_of(precision, 64), d_screen_slots, d_items + n_narrow,
                              n_wide, err, num_sms, s);
  return e;
}

int BatchPlan::kernels_per_iteration() const {
  int k = 1;   // begin
  for (int p = 0; p < kPasses; ++p)
    if (p != kPassFrameMax) k += (int)groups[p].size();   // the max pass is not launched
  if (is_screen_prec(precision)) k += (n_items > n_wide ? 1 : 0) + (n_wide ? 1 : 0) + 6;
  else k += 2;
  k += (int)large.size() * (is_screen_prec(precision) ? 4 : 2);
  return k;
}

}  // namespace trstmi
