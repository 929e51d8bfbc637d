// plan_io.cu -- plan checkpoint: the prepared tables (keys, directories,
// trained models, learned windows), value grids and tuning choices written
// to a versioned binary file and read back; a loaded plan gives the same
// results as the one that was saved.  The prepared tables are read whole on
// the host and their layout checked there before anything reaches the
// device; value grids follow in chunks.
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "plan.h"
#include "plan_host.h"

using namespace ss;

namespace {

constexpr char kMagic[8] = {'S', 'S', 'P', 'L', 'A', 'N', 0, 1};
constexpr int32_t kVersion = 11;

struct Writer {
  FILE* f;
  bool ok = true;
  void raw(const void* p, size_t n) { ok = ok && fwrite(p, 1, n, f) == n; }
  template <class T> void val(const T& v) { raw(&v, sizeof(T)); }
  template <class T> void vec(const std::vector<T>& v) {
    val<int64_t>((int64_t)v.size());
    if (!v.empty()) raw(v.data(), v.size() * sizeof(T));
  }
};

struct Reader {
  FILE* f;
  bool ok = true;
  void raw(void* p, size_t n) { ok = ok && fread(p, 1, n, f) == n; }
  template <class T> void val(T& v) { raw(&v, sizeof(T)); }
  template <class T> void vec(std::vector<T>& v) {
    int64_t n = 0;
    val(n);
    if (!ok || n < 0 || n > (int64_t)1 << 34) { ok = false; return; }
    v.resize((size_t)n);
    if (n) raw(v.data(), (size_t)n * sizeof(T));
  }
};

ss_status copy_out(Writer& w, const void* dptr, int64_t bytes) {
  std::vector<unsigned char> buf((size_t)std::min<int64_t>(bytes, (int64_t)64 << 20));
  for (int64_t o = 0; o < bytes; o += (int64_t)buf.size()) {
    const int64_t n = std::min<int64_t>((int64_t)buf.size(), bytes - o);
    SS_CHECK_CUDA(cudaMemcpy(buf.data(), (const unsigned char*)dptr + o, (size_t)n, cudaMemcpyDeviceToHost));
    w.raw(buf.data(), (size_t)n);
  }
  return SS_OK;
}

// Largest bucket of a directory of nb + 1 counts over `count` keys: counts
// start at 0, never decrease and end at `count`; -1 when they do not.
template <class D>
int dir_occupancy(const D* d, int nb, int count) {
  if ((int64_t)d[0] != 0 || (int64_t)d[nb] != count) return -1;
  int occ = 0;
  for (int b = 0; b < nb; ++b) {
    if ((int64_t)d[b + 1] < (int64_t)d[b]) return -1;
    occ = std::max(occ, (int)((int64_t)d[b + 1] - (int64_t)d[b]));
  }
  return occ;
}

// Host-side layout checks of a plan read from a file, made before any kernel
// sees it.  The blob offsets must be those plan creation gives for the
// recorded sizes and directory budgets; in every blob, each header field that
// places or sizes an access (geometry, Eytzinger depth, ballot stride, bucket
// directories with their cuts and occupancies, the fine directory over all
// keys, the wide section) must agree with that geometry and with the blob's
// own directories.  Returns nullptr, or what is wrong.
const char* check_layout(const ss_plan* p, const std::vector<unsigned char>& hb) {
  const int nblobs = p->kind == 1 ? p->ntables : 2 * p->ntables;
  const bool cells = p->kind == 2;
  int64_t off = 0;
  for (int j = 0; j < nblobs; ++j) {
    const int n = p->kind == 1 ? p->sizes[j] : (j & 1) ? p->sizes_t[j / 2] : p->sizes[j / 2];
    if (n < 2 || n > (cells ? (1 << 20) : (1 << 30))) return "table size out of range";
    if (p->dir_cap[j] < 1 || p->dir_cap[j] > SS_MAX_DIR_CAP) return "directory budget out of range";
    if (p->algo[j] < 0 || p->algo[j] >= BL_NUM) return "unknown algorithm";
    if (p->blob_off[j] != off) return "blob offsets do not follow the layout";
    off += (blob_geom_dev(n, p->dir_cap[j], cells).bytes + 255) & ~(int64_t)255;
  }
  if (off != p->blob_bytes || (int64_t)hb.size() != off) return "blob bytes do not follow the layout";
  for (int j = 0; j < nblobs; ++j) {
    const int n = p->kind == 1 ? p->sizes[j] : (j & 1) ? p->sizes_t[j / 2] : p->sizes[j / 2];
    const int nk = n - 1;
    const BlobGeom g = blob_geom_dev(n, p->dir_cap[j], cells);
    const unsigned char* blob = hb.data() + p->blob_off[j];
    BlobHdr h;
    std::memcpy(&h, blob, sizeof(h));
    if (h.n != n || h.nk != nk || h.ns != g.ns || h.stride != g.stride || h.D != g.D || h.dir_cap != p->dir_cap[j] ||
        h.off_mlp != g.off_mlp || h.off_dir != g.off_dir || h.off_keys != g.off_keys || h.off_eyt != g.off_eyt ||
        h.staged_end != g.staged_end || h.off_full != g.off_full || h.off_cells != g.off_cells)
      return "blob header does not match its geometry";
    if (h.algo != p->algo[j] || (h.algo == BL_WIDE && g.off_wide < 0)) return "blob algorithm does not match the plan";
    const int G = h.algo == BL_BALLOT8 ? 8 : h.algo == BL_BALLOT16 ? 16 : 32;
    int S0 = 1;
    while ((int64_t)S0 * (G + 1) < (int64_t)g.ns + 1) S0 *= (G + 1);
    if (h.S0 != S0) return "ballot stride does not match the table";
    if (h.shift < 0 || h.shift > 63 || h.nb < 1 || h.nb > h.dir_cap) return "bucket directory out of range";
    std::vector<uint16_t> dir((size_t)h.nb + 1);
    std::memcpy(dir.data(), blob + g.off_dir, dir.size() * sizeof(uint16_t));
    if (dir_occupancy(dir.data(), h.nb, g.ns) != h.occ) return "bucket directory or occupancy inconsistent";
    if (h.E < 0) return "negative learned window";
    if (g.stride > 1) {
      if (h.gshift < 0 || h.gshift > 63 || h.gnb < 1 || h.gnb > fine_dir_cap(nk)) return "fine directory out of range";
      std::vector<int32_t> gdir((size_t)h.gnb + 1);
      std::memcpy(gdir.data(), blob + g.off_full + (int64_t)(nk + kPad) * 8, gdir.size() * sizeof(int32_t));
      if (dir_occupancy(gdir.data(), h.gnb, nk) < 0) return "fine directory inconsistent";
    } else if (h.gnb != 0) {
      return "fine directory on a table staged whole";
    }
    if (g.off_wide >= 0) {
      const WideGeom wg = wide_geom(nk);
      WideHdr w;
      std::memcpy(&w, blob + g.off_wide, sizeof(w));
      if (w.L != wg.L || w.dcap != wg.dcap || w.off_dir != wg.off_dir || w.off_samples != wg.off_samples ||
          w.off_shift != wg.off_shift || w.off_leaf != wg.off_leaf || w.shift < 0 || w.shift > 63 || w.nb < 1 ||
          w.nb > w.dcap)
        return "wide section header does not match its geometry";
      std::vector<uint16_t> wdir((size_t)w.nb + 1);
      std::memcpy(wdir.data(), blob + g.off_wide + wg.off_dir, wdir.size() * sizeof(uint16_t));
      if (dir_occupancy(wdir.data(), w.nb, wg.L) != w.occ) return "wide directory or occupancy inconsistent";
      for (int s2 = 0; s2 < wg.L; ++s2) {
        const uint8_t sh = blob[g.off_wide + wg.off_shift + s2];
        uint16_t last;                     // slot 15 of leaf s2: offsets 8..15 sit after all leaves' 0..7
        std::memcpy(&last, blob + g.off_wide + wg.off_leaf + ((int64_t)(wg.L + s2) * (kLeaf / 2) + kLeaf / 2 - 1) * 2,
                    sizeof(last));
        if (sh > 63 || last != sh) return "wide leaf shift out of range";
      }
    }
  }
  for (int b = 0; b < kNumBuckets; ++b)
    if (p->bucket_algo[b] < 0 || p->bucket_algo[b] >= BL_NUM || !(p->bucket_mult[b] > 0.0f && p->bucket_mult[b] < 1e6f) ||
        p->bucket_tables[b] < 0)
      return "tuning choices out of range";
  return nullptr;
}

ss_status copy_in(Reader& r, void* dptr, int64_t bytes) {
  std::vector<unsigned char> buf((size_t)std::min<int64_t>(std::max<int64_t>(bytes, 1), (int64_t)64 << 20));
  for (int64_t o = 0; o < bytes; o += (int64_t)buf.size()) {
    const int64_t n = std::min<int64_t>((int64_t)buf.size(), bytes - o);
    r.raw(buf.data(), (size_t)n);
    if (!r.ok) return fail(SS_EINVAL, "ss_plan_load: truncated file");
    SS_CHECK_CUDA(cudaMemcpy((unsigned char*)dptr + o, buf.data(), (size_t)n, cudaMemcpyHostToDevice));
  }
  return SS_OK;
}

}  // namespace

extern "C" ss_status ss_plan_save(const ss_plan* p, const char* path) {
  if (p == nullptr || path == nullptr) return fail(SS_EINVAL, "ss_plan_save: null pointer");
  FILE* f = std::fopen(path, "wb");
  if (f == nullptr) return fail(SS_EINVAL, std::string("ss_plan_save: cannot open ") + path);
  Writer w{f};
  w.raw(kMagic, 8);
  w.val(kVersion);
  w.val<int32_t>(p->kind);
  w.val<int32_t>(p->ntables);
  ss_plan_opts o = p->opts;
  o.tune_cache = nullptr;
  w.val(o);
  w.vec(p->sizes);
  w.vec(p->sizes_t);
  w.vec(p->X_off);
  w.vec(p->dir_cap);
  w.vec(p->algo);
  w.vec(p->blob_off);
  w.vec(p->grid_off);
  w.raw(p->bucket_algo, sizeof(p->bucket_algo));
  w.raw(p->bucket_mult, sizeof(p->bucket_mult));
  w.raw(p->bucket_tables, sizeof(p->bucket_tables));
  w.val<int32_t>(p->tuned);
  w.val<int64_t>(p->blob_bytes);
  ss_status st = copy_out(w, p->d_blobs, p->blob_bytes);
  const int64_t gcount = p->kind == 2 ? p->grid_off.back() : 0;
  const int64_t ccount = p->kind == 2 ? 4 * p->cell_off.back() : 0;     // float-float corners
  if (st == SS_OK && p->kind == 2) {
    w.val<int64_t>(ccount);
    st = copy_out(w, p->d_grid, ccount * (int64_t)sizeof(float2));
    const int32_t has64 = p->d_grid64 != nullptr;
    w.val(has64);
    if (st == SS_OK && has64) st = copy_out(w, p->d_grid64, gcount * (int64_t)sizeof(double));
  }
  const bool ok = w.ok;
  std::fclose(f);
  if (st != SS_OK) return st;
  return ok ? SS_OK : fail(SS_EINVAL, "ss_plan_save: write failed");
}

extern "C" ss_status ss_plan_load(ss_plan** out, const char* path, cudaStream_t stream) {
  if (out == nullptr || path == nullptr) return fail(SS_EINVAL, "ss_plan_load: null pointer");
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (f == nullptr) return fail(SS_EINVAL, std::string("ss_plan_load: cannot open ") + path);
  std::unique_ptr<FILE, int (*)(FILE*)> guard(f, std::fclose);
  Reader r{f};
  char magic[8];
  r.raw(magic, 8);
  int32_t ver = 0, kind = 0, ntables = 0;
  r.val(ver);
  r.val(kind);
  r.val(ntables);
  if (!r.ok || std::memcmp(magic, kMagic, 8) != 0 || ver != kVersion || (kind != 1 && kind != 2) || ntables < 1)
    return fail(SS_EINVAL, "ss_plan_load: not a plan file of this version");
  auto* p = new ss_plan();
  p->kind = kind;
  p->ntables = ntables;
  r.val(p->opts);
  p->opts.tune_cache = nullptr;
  r.vec(p->sizes);
  r.vec(p->sizes_t);
  r.vec(p->X_off);
  r.vec(p->dir_cap);
  r.vec(p->algo);
  r.vec(p->blob_off);
  r.vec(p->grid_off);
  r.raw(p->bucket_algo, sizeof(p->bucket_algo));
  r.raw(p->bucket_mult, sizeof(p->bucket_mult));
  r.raw(p->bucket_tables, sizeof(p->bucket_tables));
  r.val(p->tuned);
  r.val(p->blob_bytes);
  const size_t nblobs = (size_t)(kind == 1 ? ntables : 2 * ntables);
  if (!r.ok || p->sizes.size() != (size_t)ntables || p->blob_off.size() != nblobs || p->algo.size() != nblobs ||
      p->dir_cap.size() != nblobs || p->blob_bytes <= 0 ||
      p->sizes_t.size() != (size_t)(kind == 2 ? ntables : 0) ||
      p->X_off.size() != (size_t)(kind == 1 ? ntables + 1 : 2 * (ntables + 1)) ||
      (kind == 2 && p->grid_off.size() != (size_t)ntables + 1)) {
    delete p;
    return fail(SS_EINVAL, "ss_plan_load: corrupt plan file");
  }
  if (kind == 2) {
    bool ok = p->grid_off[0] >= 0;
    for (int k = 0; ok && k < ntables; ++k)
      ok = p->sizes[k] >= 2 && p->sizes_t[k] >= 2 && p->sizes[k] <= (1 << 20) && p->sizes_t[k] <= (1 << 20) &&
           p->grid_off[k + 1] - p->grid_off[k] == (int64_t)p->sizes[k] * p->sizes_t[k];
    if (!ok) {
      delete p;
      return fail(SS_EINVAL, "ss_plan_load: corrupt plan file (table sizes or value offsets)");
    }
  }
  if (ss_status s0 = check_plan_opts(p->opts, kind)) {
    delete p;
    return fail(s0, std::string("ss_plan_load: ") + ss_last_error());
  }
  ss_status st = [&]() -> ss_status {
    // the prepared tables pass the layout checks on the host before they are copied to the device
    if (p->blob_bytes > ((int64_t)1 << 40)) return fail(SS_EINVAL, "ss_plan_load: corrupt plan file (blob bytes)");
    std::vector<unsigned char> hb((size_t)p->blob_bytes);
    r.raw(hb.data(), hb.size());
    if (!r.ok) return fail(SS_EINVAL, "ss_plan_load: truncated file");
    if (const char* why = check_layout(p, hb)) return fail(SS_EINVAL, std::string("ss_plan_load: corrupt plan file (") + why + ")");
    if (cudaMalloc(&p->d_blobs, p->blob_bytes) != cudaSuccess) return fail(SS_ENOMEM, "ss_plan_load: device allocation failed");
    SS_CHECK_CUDA(cudaMemcpy(p->d_blobs, hb.data(), hb.size(), cudaMemcpyHostToDevice));
    SS_CHECK_CUDA(cudaMalloc(&p->d_blob_off, nblobs * sizeof(int64_t)));
    SS_CHECK_CUDA(cudaMemcpy(p->d_blob_off, p->blob_off.data(), nblobs * sizeof(int64_t), cudaMemcpyHostToDevice));
    p->device_bytes = p->blob_bytes;
    if (kind == 2) {
      plan_cell_offsets(p);
      const int64_t gcount = p->grid_off.back();
      int64_t ccount = 0;
      r.val(ccount);
      if (!r.ok || ccount != 4 * p->cell_off.back()) return fail(SS_EINVAL, "ss_plan_load: corrupt plan file");
      if (cudaMalloc(&p->d_grid, std::max<int64_t>(ccount, 1) * sizeof(float2)) != cudaSuccess)
        return fail(SS_ENOMEM, "ss_plan_load: device allocation failed");
      if (ss_status s2 = copy_in(r, p->d_grid, ccount * (int64_t)sizeof(float2))) return s2;
      int32_t has64 = 0;
      r.val(has64);
      if (has64) {
        if (cudaMalloc(&p->d_grid64, gcount * sizeof(double)) != cudaSuccess)
          return fail(SS_ENOMEM, "ss_plan_load: device allocation failed");
        if (ss_status s2 = copy_in(r, p->d_grid64, gcount * (int64_t)sizeof(double))) return s2;
      }
      SS_CHECK_CUDA(cudaMalloc(&p->d_grid_off, (ntables + 1) * sizeof(int64_t)));
      SS_CHECK_CUDA(cudaMemcpy(p->d_grid_off, p->grid_off.data(), (ntables + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
      SS_CHECK_CUDA(cudaMalloc(&p->d_cell_off, (ntables + 1) * sizeof(int64_t)));
      SS_CHECK_CUDA(cudaMemcpy(p->d_cell_off, p->cell_off.data(), (ntables + 1) * sizeof(int64_t), cudaMemcpyHostToDevice));
      p->device_bytes += ccount * (int64_t)sizeof(float2) + (has64 ? gcount * (int64_t)sizeof(double) : 0);
    }
    return plan_window_stats(p);
  }();
  (void)stream;
  if (st != SS_OK) {
    delete p;
    return st;
  }
  *out = p;
  return SS_OK;
}
