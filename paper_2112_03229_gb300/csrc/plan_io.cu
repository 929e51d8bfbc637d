// plan_io.cu -- plan checkpoint: the prepared tables (keys, directories,
// trained models, learned windows), value grids and tuning choices written
// to a versioned binary file and read back; a loaded plan gives the same
// results as the one that was saved.
#include <cstdio>
#include <cstring>
#include <memory>
#include <vector>

#include "plan.h"
#include "plan_host.h"

using namespace ss;

namespace {

constexpr char kMagic[8] = {'S', 'S', 'P', 'L', 'A', 'N', 0, 1};
constexpr int32_t kVersion = 9;

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
      p->dir_cap.size() != nblobs || p->blob_bytes <= 0 || (kind == 2 && p->grid_off.size() != (size_t)ntables + 1)) {
    delete p;
    return fail(SS_EINVAL, "ss_plan_load: corrupt plan file");
  }
  ss_status st = [&]() -> ss_status {
    if (cudaMalloc(&p->d_blobs, p->blob_bytes) != cudaSuccess) return fail(SS_ENOMEM, "ss_plan_load: device allocation failed");
    if (ss_status s2 = copy_in(r, p->d_blobs, p->blob_bytes)) return s2;
    SS_CHECK_CUDA(cudaMalloc(&p->d_blob_off, nblobs * sizeof(int64_t)));
    SS_CHECK_CUDA(cudaMemcpy(p->d_blob_off, p->blob_off.data(), nblobs * sizeof(int64_t), cudaMemcpyHostToDevice));
    p->device_bytes = p->blob_bytes;
    if (kind == 2) {
      if (p->sizes_t.size() != (size_t)ntables) return fail(SS_EINVAL, "ss_plan_load: corrupt plan file");
      for (int k = 0; k < ntables; ++k)
        if (p->sizes[k] < 2 || p->sizes_t[k] < 2) return fail(SS_EINVAL, "ss_plan_load: corrupt plan file");
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
