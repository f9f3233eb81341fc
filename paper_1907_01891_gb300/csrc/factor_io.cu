// factor_io.cu -- a factor written to a file and read back.
//
// The paper factors A once and keeps the result so that every later batch of
// slices is solved with it ("computed just once and, by storing the
// results...", Sec. II-B); its factor lives on disk as tile files.  Here a
// factor (the factored matrix, tau, the panel T blocks and, for two-level
// factors, the per-outer-block V^T V and T) goes to one file with a header
// that records its shape, panel width, arithmetic and a caller-chosen tag
// (e.g. ct_geometry_hash of the scan it factors), and a checksum of every
// payload byte.
//
// File layout (little-endian, as the host writes it):
//   header (struct FileHeader, 128 bytes), then the payload sections in this
//   order, each a plain array: F (m x n column-major, leading dimension m,
//   element type `store`), tau (n doubles), T (npanels * nb * nb doubles),
//   and when has_blocks: Gblk and Tblk (nblocks * 128 * 128 floats each).
// The checksum is FNV-1a (64 bit) over the payload bytes in file order.
//
// Device <-> file copies go through a page-locked staging buffer of
// kStage bytes, one chunk at a time (the chunk's device copy and the file
// access alternate; nothing else is allocated on the host).
#include <errno.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "internal.cuh"

namespace ctqr {
namespace {

constexpr char kMagic[8] = {'C', 'T', 'Q', 'R', 'F', 'A', 'C', '1'};
constexpr uint32_t kVersion = 1;
constexpr size_t kStage = (size_t)64 << 20;

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t m, n;
  int32_t nb;
  int32_t prec;       // ct_prec
  int32_t store;      // ct_dtype of F
  int32_t has_blocks; // Gblk / Tblk sections present
  uint64_t tag;       // caller's tag (e.g. geometry hash), 0 = none
  uint64_t payload_bytes;
  uint64_t checksum;  // FNV-1a 64 of the payload
  uint8_t reserved[128 - 8 - 4 - 4 - 16 - 16 - 8 - 8 - 8];
};
static_assert(sizeof(FileHeader) == 128, "header layout");

constexpr uint64_t kFnvOffset = 1469598103934665603ull, kFnvPrime = 1099511628211ull;

uint64_t fnv1a(uint64_t h, const unsigned char* p, size_t n) {
  for (size_t i = 0; i < n; ++i) {
    h ^= p[i];
    h *= kFnvPrime;
  }
  return h;
}

struct Section {
  void* dev;       // device base
  int64_t rows;    // elements per column copied (contiguous in the file)
  int64_t ld;      // device leading dimension (elements)
  int64_t cols;
  size_t elem;
};

int64_t nblocks_of(const ct_factor* f) { return (f->n + 127) / 128; }

std::vector<Section> sections(const ct_factor* f, bool blocks) {
  std::vector<Section> s;
  s.push_back({f->F, f->m, f->ld, f->n, (size_t)(f->store == CT_F64 ? 8 : 4)});
  s.push_back({f->tau, f->n, f->n, 1, 8});
  const int64_t tcount = npanels(f) * f->nb * f->nb;
  s.push_back({f->T, tcount, tcount, 1, 8});
  if (blocks) {
    const int64_t bcount = nblocks_of(f) * 128 * 128;
    s.push_back({f->Gblk, bcount, bcount, 1, 4});
    s.push_back({f->Tblk, bcount, bcount, 1, 4});
  }
  return s;
}

uint64_t payload_bytes(const std::vector<Section>& secs) {
  uint64_t b = 0;
  for (const auto& x : secs) b += (uint64_t)x.rows * x.cols * x.elem;
  return b;
}

struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

struct File {
  FILE* fp = nullptr;
  ~File() {
    if (fp) fclose(fp);
  }
};

// Copy a section between the device and the file in chunks of whole column
// pieces through the staging buffer.  to_file: device -> file, else
// file -> device.  *h accumulates the checksum.
ct_status stream_section(const Section& x, FILE* fp, void* stage, bool to_file, uint64_t* h, cudaStream_t s) {
  const size_t col_bytes = (size_t)x.rows * x.elem;
  for (int64_t c = 0; c < x.cols; ++c) {
    for (size_t off = 0; off < col_bytes; off += kStage) {
      const size_t len = col_bytes - off < kStage ? col_bytes - off : kStage;
      char* dev = (char*)x.dev + (size_t)c * x.ld * x.elem + off;
      if (to_file) {
        CT_CUDA_TRY(cudaMemcpyAsync(stage, dev, len, cudaMemcpyDeviceToHost, s));
        CT_CUDA_TRY(cudaStreamSynchronize(s));
        *h = fnv1a(*h, (const unsigned char*)stage, len);
        if (fwrite(stage, 1, len, fp) != len) return CT_ERR_INVALID;
      } else {
        // the previous chunk's copy out of the staging buffer must be done
        CT_CUDA_TRY(cudaStreamSynchronize(s));
        if (fread(stage, 1, len, fp) != len) return CT_ERR_INVALID;
        *h = fnv1a(*h, (const unsigned char*)stage, len);
        CT_CUDA_TRY(cudaMemcpyAsync(dev, stage, len, cudaMemcpyHostToDevice, s));
      }
    }
  }
  return CT_OK;
}

// Read and check a header; CT_ERR_INVALID for anything malformed.
ct_status read_header(FILE* fp, FileHeader* hd) {
  if (fread(hd, 1, sizeof(*hd), fp) != sizeof(*hd)) return CT_ERR_INVALID;
  if (memcmp(hd->magic, kMagic, 8) != 0 || hd->version != kVersion || hd->header_bytes != sizeof(*hd))
    return CT_ERR_INVALID;
  if (hd->n < 1 || hd->m < hd->n || hd->nb < 1 || hd->nb > 64) return CT_ERR_INVALID;
  if (hd->prec != CT_PREC_F64 && hd->prec != CT_PREC_F32 && !tc_prec((ct_prec)hd->prec)) return CT_ERR_INVALID;
  if (hd->store != (hd->prec == CT_PREC_F64 ? CT_F64 : CT_F32)) return CT_ERR_INVALID;
  if (hd->has_blocks != (tc_prec((ct_prec)hd->prec) ? 1 : 0)) return CT_ERR_INVALID;
  return CT_OK;
}

}  // namespace
}  // namespace ctqr

using namespace ctqr;

extern "C" {

uint64_t ct_geometry_hash(const ct_geometry* g, double lambda) {
  if (!g) return 0;
  uint64_t h = kFnvOffset;
  auto mix_i = [&](int64_t v) { h = fnv1a(h, (const unsigned char*)&v, sizeof(v)); };
  auto mix_d = [&](double v) {
    if (v == 0.0) v = 0.0;  // +0 and -0 hash alike
    h = fnv1a(h, (const unsigned char*)&v, sizeof(v));
  };
  mix_i(g->beam);
  mix_i(g->nx);
  mix_i(g->ny);
  mix_d(g->pixel);
  mix_i(g->n_views);
  mix_i(g->n_bins);
  mix_d(g->angle0);
  mix_d(g->angle_span);
  mix_d(g->src_iso);
  mix_d(g->det_span);
  mix_i(g->angle_rule);
  mix_d(lambda);
  return h == 0 ? 1 : h;
}

ct_status ct_factor_save(const ct_factor* f, const char* path, uint64_t tag, void* stream) {
  if (!f || !path || !*path) return CT_ERR_INVALID;
  if (f->F_host) return CT_ERR_UNSUPPORTED;  // the caller already holds it in host memory
  cudaStream_t s = (cudaStream_t)stream;
  const bool blocks = f->Gblk && f->Tblk;
  const auto secs = sections(f, blocks);
  FileHeader hd;
  memset(&hd, 0, sizeof(hd));
  memcpy(hd.magic, kMagic, 8);
  hd.version = kVersion;
  hd.header_bytes = sizeof(hd);
  hd.m = f->m;
  hd.n = f->n;
  hd.nb = f->nb;
  hd.prec = f->prec;
  hd.store = f->store;
  hd.has_blocks = blocks ? 1 : 0;
  hd.tag = tag;
  hd.payload_bytes = payload_bytes(secs);
  File out;
  out.fp = fopen(path, "wb");
  if (!out.fp) return CT_ERR_INVALID;
  // header first with a zero checksum, rewritten once the payload is summed
  if (fwrite(&hd, 1, sizeof(hd), out.fp) != sizeof(hd)) return CT_ERR_INVALID;
  Pinned stage;
  CT_CUDA_TRY(cudaMallocHost(&stage.p, kStage));
  uint64_t h = kFnvOffset;
  for (const auto& x : secs) {
    ct_status st = stream_section(x, out.fp, stage.p, true, &h, s);
    if (st != CT_OK) return st;
  }
  hd.checksum = h;
  if (fseek(out.fp, 0, SEEK_SET) != 0 || fwrite(&hd, 1, sizeof(hd), out.fp) != sizeof(hd)) return CT_ERR_INVALID;
  if (fclose(out.fp) != 0) {
    out.fp = nullptr;
    return CT_ERR_INVALID;
  }
  out.fp = nullptr;
  return CT_OK;
}

ct_status ct_factor_file_info(const char* path, int64_t* m, int64_t* n, int* nb, ct_prec* prec, uint64_t* tag) {
  if (!path) return CT_ERR_INVALID;
  File in;
  in.fp = fopen(path, "rb");
  if (!in.fp) return CT_ERR_INVALID;
  FileHeader hd;
  ct_status st = read_header(in.fp, &hd);
  if (st != CT_OK) return st;
  if (m) *m = hd.m;
  if (n) *n = hd.n;
  if (nb) *nb = hd.nb;
  if (prec) *prec = (ct_prec)hd.prec;
  if (tag) *tag = hd.tag;
  return CT_OK;
}

ct_status ct_factor_load(const char* path, ct_factor** out, uint64_t* tag, void* stream) {
  if (!out) return CT_ERR_INVALID;
  *out = nullptr;
  if (!path) return CT_ERR_INVALID;
  File in;
  in.fp = fopen(path, "rb");
  if (!in.fp) return CT_ERR_INVALID;
  FileHeader hd;
  ct_status st = read_header(in.fp, &hd);
  if (st != CT_OK) return st;
  // the file must hold exactly the payload the header describes
  {
    ct_factor shape;
    shape.m = hd.m;
    shape.n = hd.n;
    shape.ld = hd.m;
    shape.nb = hd.nb;
    shape.store = (ct_dtype)hd.store;
    shape.F = nullptr;
    const uint64_t want = payload_bytes(sections(&shape, hd.has_blocks != 0));
    if (want != hd.payload_bytes) return CT_ERR_INVALID;
    if (fseek(in.fp, 0, SEEK_END) != 0) return CT_ERR_INVALID;
    const long size = ftell(in.fp);
    if (size < 0 || (uint64_t)size != sizeof(hd) + want) return CT_ERR_INVALID;
    if (fseek(in.fp, (long)sizeof(hd), SEEK_SET) != 0) return CT_ERR_INVALID;
  }
  cudaStream_t s = (cudaStream_t)stream;
  DeviceInfo di;
  if ((st = device_info(&di)) != CT_OK) return st;
  ct_factor* f = new ct_factor;
  f->m = hd.m;
  f->n = hd.n;
  f->nb = hd.nb;
  f->prec = (ct_prec)hd.prec;
  f->store = (ct_dtype)hd.store;
  f->device = di.device;
  if ((st = alloc_factor_matrix(f)) != CT_OK || (st = alloc_factor_aux(f, di)) != CT_OK) {
    free_factor(f);
    return st;
  }
  if (cudaMemsetAsync(f->status, 0, sizeof(int), s) != cudaSuccess) {
    cudaGetLastError();
    free_factor(f);
    return CT_ERR_CUDA;
  }
  Pinned stage;
  if (cudaMallocHost(&stage.p, kStage) != cudaSuccess) {
    cudaGetLastError();
    free_factor(f);
    return CT_ERR_NOMEM;
  }
  uint64_t h = kFnvOffset;
  for (const auto& x : sections(f, hd.has_blocks != 0)) {
    if ((st = stream_section(x, in.fp, stage.p, false, &h, s)) != CT_OK) {
      cudaStreamSynchronize(s);
      free_factor(f);
      return st;
    }
  }
  if (cudaStreamSynchronize(s) != cudaSuccess) {
    cudaGetLastError();
    free_factor(f);
    return CT_ERR_CUDA;
  }
  if (h != hd.checksum) {
    free_factor(f);
    return CT_ERR_INVALID;
  }
  if (tag) *tag = hd.tag;
  *out = f;
  return CT_OK;
}

}  // extern "C"
