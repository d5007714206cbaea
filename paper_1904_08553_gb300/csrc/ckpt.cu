// ckpt.cu -- checkpoint / resume of a context (dcd_save, dcd_load) and of a
// learned-screen network (dcd_mlp_save, dcd_mlp_load).  The paper has no
// counterpart: it runs each input stream start to finish.  What a resumed
// context needs is what the next step of Sec. III-D reads: G_{t-1} (the CSR),
// C_{t-1} (the labels) and the step counter t, plus the mode, the
// configuration, the degree-bin plan and the last R_t (for dcd_get_rset).
//
// File layout (little-endian, every section padded with zeros to a multiple
// of 8 bytes):
//   CkptHeader (256 bytes)
//   row_ptr   (n + 1) int64
//   col       nnz int32
//   w         nnz int32
//   labels    n int32
//   rset      n uint8            (when kFlagRset is set)
//   checksum  uint64: FNV-1a over the 64-bit words of everything before it
//
// The arrays move through a pinned host buffer in chunks, so a graph of any
// size needs only that buffer on the host (plus row_ptr when loading, which
// the entry checks walk).  Loading checks every value on the host before it
// reaches the device: a damaged or foreign file fails with DCD_EINVAL and
// never becomes an out-of-range index in a kernel.
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "prims.cuh"
#include "state.cuh"

namespace dcd {
namespace {

constexpr char kMagic[8] = {'D', 'C', 'D', 'C', 'K', 'P', 'T', '1'};
constexpr char kMlpMagic[8] = {'D', 'C', 'D', 'M', 'L', 'P', '0', '1'};
constexpr uint32_t kVersion = 1;
constexpr uint32_t kFlagRset = 1u;
constexpr size_t kChunk = (size_t)32 << 20;  // bytes per staging transfer (a multiple of 8)

struct CkptHeader {
  char magic[8];
  uint32_t version;
  uint32_t flags;
  int64_t n;
  int64_t nnz;
  int64_t t;
  int32_t mode;
  int32_t nb;
  dcd_config cfg;
  int32_t var[kMaxBins];
  int64_t hi[kMaxBins];  // -1 for the last (unbounded) bin
};
static_assert(sizeof(dcd_config) == 64, "config layout");
static_assert(offsetof(CkptHeader, cfg) == 48 && offsetof(CkptHeader, var) == 112 && offsetof(CkptHeader, hi) == 160,
              "header layout");
static_assert(sizeof(CkptHeader) == 256, "header size");

struct Fnv {
  uint64_t h = 1469598103934665603ull;
  void words(const void* p, size_t bytes) {  // bytes is a multiple of 8
    const unsigned char* b = static_cast<const unsigned char*>(p);
    for (size_t i = 0; i < bytes; i += 8) {
      uint64_t x;
      memcpy(&x, b + i, 8);
      h = (h ^ x) * 1099511628211ull;
    }
  }
};

constexpr size_t pad8(size_t b) { return (b + 7) & ~(size_t)7; }

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

struct Pinned {
  unsigned char* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

// device -> file, through the staging buffer; pads the section to 8 bytes
int save_section(FILE* f, Fnv* fnv, const void* dev, size_t bytes, unsigned char* stage, cudaStream_t s) {
  const unsigned char* d = static_cast<const unsigned char*>(dev);
  const size_t padded = pad8(bytes);
  for (size_t off = 0; off < padded; off += kChunk) {
    const size_t len = padded - off < kChunk ? padded - off : kChunk;
    const size_t real = off < bytes ? (bytes - off < len ? bytes - off : len) : 0;
    if (real) DCD_TRY_CUDA(cudaMemcpyAsync(stage, d + off, real, cudaMemcpyDeviceToHost, s));
    DCD_TRY_CUDA(cudaStreamSynchronize(s));
    memset(stage + real, 0, len - real);
    fnv->words(stage, len);
    if (fwrite(stage, 1, len, f) != len) return DCD_EIO;
  }
  return DCD_OK;
}

// Reads one padded section chunk by chunk.  check(stage, first_element,
// count) validates the chunk's elements on the host before the copy to the
// device; the padding must be zero.
template <typename T, typename Check>
int load_section(FILE* f, Fnv* fnv, T* dev, size_t count, unsigned char* stage, cudaStream_t s, Check check) {
  const size_t bytes = count * sizeof(T), padded = pad8(bytes);
  static_assert(kChunk % sizeof(T) == 0, "chunks hold whole elements");
  for (size_t off = 0; off < padded; off += kChunk) {
    const size_t len = padded - off < kChunk ? padded - off : kChunk;
    const size_t real = off < bytes ? (bytes - off < len ? bytes - off : len) : 0;
    if (fread(stage, 1, len, f) != len) return DCD_EINVAL;  // truncated
    fnv->words(stage, len);
    for (size_t x = real; x < len; x++)
      if (stage[x]) return DCD_EINVAL;
    if (!check(reinterpret_cast<const T*>(stage), off / sizeof(T), real / sizeof(T))) return DCD_EINVAL;
    if (real) {
      DCD_TRY_CUDA(cudaMemcpyAsync(reinterpret_cast<unsigned char*>(dev) + off, stage, real, cudaMemcpyHostToDevice, s));
      DCD_TRY_CUDA(cudaStreamSynchronize(s));
    }
  }
  return DCD_OK;
}

int read_header(FILE* f, CkptHeader* h) {
  if (fread(h, 1, sizeof(*h), f) != sizeof(*h)) return DCD_EINVAL;
  if (memcmp(h->magic, kMagic, 8) != 0 || h->version != kVersion || (h->flags & ~kFlagRset)) return DCD_EINVAL;
  if (h->n <= 0 || h->n > INT32_MAX || h->nnz < 0 || h->t < 0) return DCD_EINVAL;
  // a level-0 row holds at most n - 1 entries (no self-loops, no repeats),
  // and every undirected edge is stored in both of its rows
  if (h->nnz > h->n * (h->n - 1) || (h->nnz & 1)) return DCD_EINVAL;
  if (h->mode < DCD_MODE_STATIC || h->mode > DCD_MODE_LEARNED) return DCD_EINVAL;
  if (h->nb < 1 || h->nb > kMaxBins) return DCD_EINVAL;
  return DCD_OK;
}

int save_impl(dcd_ctx* c, FILE* f) {
  cudaStream_t s = c->stream;
  CkptHeader h;
  memset(&h, 0, sizeof(h));
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.flags = c->rset.get() ? kFlagRset : 0u;
  h.n = c->n;
  h.nnz = c->nnz;
  h.t = c->t;
  h.mode = c->mode;
  h.cfg = c->cfg;
  DCD_TRY(dcd_get_bins(c, &h.nb, h.var, h.hi));
  Fnv fnv;
  fnv.words(&h, sizeof(h));
  if (fwrite(&h, 1, sizeof(h), f) != sizeof(h)) return DCD_EIO;
  Pinned stage;
  if (cudaMallocHost(&stage.p, kChunk) != cudaSuccess) return DCD_ENOMEM;
  const int k = c->cur;
  DCD_TRY(save_section(f, &fnv, c->rp[k].get(), (c->n + 1) * sizeof(int64_t), stage.p, s));
  DCD_TRY(save_section(f, &fnv, c->col[k].get(), c->nnz * sizeof(int32_t), stage.p, s));
  DCD_TRY(save_section(f, &fnv, c->w[k].get(), c->nnz * sizeof(int32_t), stage.p, s));
  DCD_TRY(save_section(f, &fnv, c->labels.get(), c->n * sizeof(int32_t), stage.p, s));
  if (h.flags & kFlagRset) DCD_TRY(save_section(f, &fnv, c->rset.get(), c->n, stage.p, s));
  if (fwrite(&fnv.h, 1, 8, f) != 8) return DCD_EIO;
  return DCD_OK;
}

int load_impl(FILE* f, const CkptHeader& h, dcd_ctx* c) {
  cudaStream_t s = c->stream;
  const int64_t n = h.n, nnz = h.nnz;
  DCD_TRY(dcd_set_bins(c, h.nb, h.var, h.hi));
  Fnv fnv;
  fnv.words(&h, sizeof(h));
  Pinned stage;
  if (cudaMallocHost(&stage.p, kChunk) != cudaSuccess) return DCD_ENOMEM;
  c->cur = 0;
  DCD_TRY(c->rp[0].ensure(&c->mem, n + 1));
  DCD_TRY(c->col[0].ensure(&c->mem, nnz > 0 ? nnz : 1));
  DCD_TRY(c->w[0].ensure(&c->mem, nnz > 0 ? nnz : 1));
  // row_ptr: starts at 0, never decreases, ends at nnz, rows below n entries
  std::vector<int64_t> rp;
  try {
    rp.resize(n + 1);
  } catch (...) {
    return DCD_ENOMEM;
  }
  DCD_TRY(load_section<int64_t>(f, &fnv, c->rp[0].get(), n + 1, stage.p, s,
                                [&](const int64_t* x, size_t i0, size_t cnt) {
                                  for (size_t j = 0; j < cnt; j++) {
                                    const size_t i = i0 + j;
                                    const int64_t v = x[j];
                                    if (i == 0 ? v != 0 : (v < rp[i - 1] || v - rp[i - 1] > n - 1)) return false;
                                    rp[i] = v;
                                  }
                                  return true;
                                }));
  if (rp[n] != nnz) return DCD_EINVAL;
  // col: in [0, n), no self-loop, strictly increasing along each row (the
  // walk's row and previous column carry over from chunk to chunk)
  int64_t row = 0;
  int64_t prev = -1;
  DCD_TRY(load_section<int32_t>(f, &fnv, c->col[0].get(), nnz, stage.p, s,
                                [&](const int32_t* x, size_t e0, size_t cnt) {
                                  for (size_t j = 0; j < cnt; j++) {
                                    const int64_t e = (int64_t)(e0 + j);
                                    while (rp[row + 1] <= e) {
                                      row++;
                                      prev = -1;
                                    }
                                    const int64_t v = x[j];
                                    if (v < 0 || v >= n || v == row || v <= prev) return false;
                                    prev = v;
                                  }
                                  return true;
                                }));
  DCD_TRY(load_section<int32_t>(f, &fnv, c->w[0].get(), nnz, stage.p, s,
                                [&](const int32_t* x, size_t, size_t cnt) {
                                  for (size_t j = 0; j < cnt; j++)
                                    if (x[j] <= 0) return false;
                                  return true;
                                }));
  DCD_TRY(load_section<int32_t>(f, &fnv, c->labels.get(), n, stage.p, s,
                                [&](const int32_t* x, size_t, size_t cnt) {
                                  for (size_t j = 0; j < cnt; j++)
                                    if (x[j] < 0 || x[j] >= n) return false;
                                  return true;
                                }));
  if (h.flags & kFlagRset)
    DCD_TRY(load_section<uint8_t>(f, &fnv, c->rset.get(), n, stage.p, s,
                                  [&](const uint8_t* x, size_t, size_t cnt) {
                                    for (size_t j = 0; j < cnt; j++)
                                      if (x[j] > 1) return false;
                                    return true;
                                  }));
  uint64_t sum = 0;
  if (fread(&sum, 1, 8, f) != 8 || sum != fnv.h) return DCD_EINVAL;
  unsigned char extra;
  if (fread(&extra, 1, 1, f) != 0) return DCD_EINVAL;  // trailing bytes
  c->nnz = nnz;
  c->t = h.t;
  c->mode = h.mode;
  return DCD_OK;
}

}  // namespace
}  // namespace dcd

using namespace dcd;

extern "C" {

int dcd_save(dcd_ctx* c, const char* path) {
  if (!c || !path || !*path) return DCD_EINVAL;
  if (c->n_ins || c->n_del) return DCD_ESTATE;
  DCD_TRY_CUDA(cudaSetDevice(c->device));
  const std::string tmp = std::string(path) + ".tmp";
  int rc;
  {
    File f;
    f.f = fopen(tmp.c_str(), "wb");
    if (!f.f) return DCD_EIO;
    rc = save_impl(c, f.f);
    if (rc == DCD_OK && fflush(f.f) != 0) rc = DCD_EIO;
    if (fclose(f.f) != 0 && rc == DCD_OK) rc = DCD_EIO;
    f.f = nullptr;
  }
  if (rc == DCD_OK && rename(tmp.c_str(), path) != 0) rc = DCD_EIO;
  if (rc != DCD_OK) remove(tmp.c_str());
  return rc;
}

int dcd_load(const char* path, void* cuda_stream, dcd_ctx** out) {
  if (!path || !out) return DCD_EINVAL;
  *out = nullptr;
  File f;
  f.f = fopen(path, "rb");
  if (!f.f) return DCD_EIO;
  CkptHeader h;
  DCD_TRY(read_header(f.f, &h));
  dcd_ctx* c = nullptr;
  DCD_TRY(dcd_create(h.n, &h.cfg, cuda_stream, &c));
  const int rc = load_impl(f.f, h, c);
  if (rc != DCD_OK) {
    dcd_destroy(c);
    return rc;
  }
  *out = c;
  return DCD_OK;
}

int dcd_get_state(const dcd_ctx* c, int64_t* n_out, int64_t* t_out, int32_t* mode_out) {
  if (!c) return DCD_EINVAL;
  if (n_out) *n_out = c->n;
  if (t_out) *t_out = c->t;
  if (mode_out) *mode_out = c->mode;
  return DCD_OK;
}

int dcd_mlp_save(dcd_mlp* mlp, const char* path) {
  if (!mlp || !path || !*path) return DCD_EINVAL;
  std::vector<float> p(DCD_MLP_PARAMS + 1, 0.f);  // + 1: pad to 8 bytes
  DCD_TRY(dcd_mlp_get_params(mlp, p.data()));
  Fnv fnv;
  const uint32_t head[2] = {kVersion, DCD_MLP_PARAMS};
  unsigned char hb[16];
  memcpy(hb, kMlpMagic, 8);
  memcpy(hb + 8, head, 8);
  fnv.words(hb, 16);
  fnv.words(p.data(), p.size() * sizeof(float));
  const std::string tmp = std::string(path) + ".tmp";
  int rc = DCD_OK;
  {
    File f;
    f.f = fopen(tmp.c_str(), "wb");
    if (!f.f) return DCD_EIO;
    if (fwrite(hb, 1, 16, f.f) != 16 || fwrite(p.data(), sizeof(float), p.size(), f.f) != p.size() ||
        fwrite(&fnv.h, 1, 8, f.f) != 8)
      rc = DCD_EIO;
    if (fclose(f.f) != 0 && rc == DCD_OK) rc = DCD_EIO;
    f.f = nullptr;
  }
  if (rc == DCD_OK && rename(tmp.c_str(), path) != 0) rc = DCD_EIO;
  if (rc != DCD_OK) remove(tmp.c_str());
  return rc;
}

int dcd_mlp_load(const char* path, void* cuda_stream, dcd_mlp** out) {
  if (!path || !out) return DCD_EINVAL;
  *out = nullptr;
  std::vector<float> p(DCD_MLP_PARAMS + 1);
  unsigned char hb[16];
  uint64_t sum = 0;
  {
    File f;
    f.f = fopen(path, "rb");
    if (!f.f) return DCD_EIO;
    unsigned char extra;
    if (fread(hb, 1, 16, f.f) != 16 || fread(p.data(), sizeof(float), p.size(), f.f) != p.size() ||
        fread(&sum, 1, 8, f.f) != 8 || fread(&extra, 1, 1, f.f) != 0)
      return DCD_EINVAL;
  }
  uint32_t head[2];
  memcpy(head, hb + 8, 8);
  if (memcmp(hb, kMlpMagic, 8) != 0 || head[0] != kVersion || head[1] != DCD_MLP_PARAMS) return DCD_EINVAL;
  Fnv fnv;
  fnv.words(hb, 16);
  fnv.words(p.data(), p.size() * sizeof(float));
  if (fnv.h != sum || p[DCD_MLP_PARAMS] != 0.f) return DCD_EINVAL;
  for (int i = 0; i < DCD_MLP_PARAMS; i++)
    if (!(p[i] == p[i]) || p[i] > 3.0e38f || p[i] < -3.0e38f) return DCD_EINVAL;  // NaN or infinite
  dcd_mlp* m = nullptr;
  DCD_TRY(dcd_mlp_create(0, cuda_stream, &m));
  const int rc = dcd_mlp_set_params(m, p.data());
  if (rc != DCD_OK) {
    dcd_mlp_destroy(m);
    return rc;
  }
  *out = m;
  return DCD_OK;
}

}  // extern "C"
