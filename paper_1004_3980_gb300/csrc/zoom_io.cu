// Dictionary and index files (checkpoint / resume) and the projection export.
//
// The paper keeps the N training pairs on disk once they are extracted
// (Sec. 2.1); a dictionary file holds every array the library stores per
// pair, so a loaded dictionary is bit-identical to the saved one.  An index
// file holds the LSH parameters and the random projections (Eq. 10); loading
// rebuilds the bucket keys and bins on the device, which gives the same keys
// and bins as the saved index.  Files are little-endian with fixed-width
// fields.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "zoom_internal.h"

namespace {

zoom_status fail(zoom_status s, const std::string& m) {
  zoom_set_error(m);
  return s;
}

constexpr char kDictMagic[8] = {'Z', 'O', 'O', 'M', 'D', 'I', 'C', 'T'};
constexpr char kIndexMagic[8] = {'Z', 'O', 'O', 'M', 'I', 'N', 'D', 'X'};
constexpr uint32_t kVersion = 1;
constexpr size_t kStage = 64u << 20;   // host staging buffer of the copies

struct DictHeader {
  char magic[8];
  uint32_t version, feature;   // feature mode (0 pixels - mean, 1 / 2 gradients)
  int64_t n;
  int32_t P, s, d, dpad, ph2, ph2pad;
  double blur_sigma;
};
struct IndexHeader {
  char magic[8];
  uint32_t version, reserved;
  int64_t n;
  int32_t d, L, k, t, cap, reserved2;
  float w, reserved3;
};

struct File {
  FILE* f = nullptr;
  File(const char* path, const char* mode) : f(fopen(path, mode)) {}
  ~File() {
    if (f) fclose(f);
  }
};

// Device -> file through the staging buffer.
bool write_dev(FILE* f, const void* dev, size_t bytes, std::vector<char>& stage, cudaStream_t st,
               std::string& why) {
  for (size_t off = 0; off < bytes; off += kStage) {
    const size_t b = bytes - off < kStage ? bytes - off : kStage;
    cudaError_t e = cudaMemcpyAsync(stage.data(), (const char*)dev + off, b, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      why = cudaGetErrorString(e);
      return false;
    }
    if (fwrite(stage.data(), 1, b, f) != b) {
      why = "write failed";
      return false;
    }
  }
  return true;
}

// File -> device through the staging buffer.
bool read_dev(FILE* f, void* dev, size_t bytes, std::vector<char>& stage, cudaStream_t st,
              std::string& why) {
  for (size_t off = 0; off < bytes; off += kStage) {
    const size_t b = bytes - off < kStage ? bytes - off : kStage;
    if (fread(stage.data(), 1, b, f) != b) {
      why = "file truncated";
      return false;
    }
    cudaError_t e = cudaMemcpyAsync((char*)dev + off, stage.data(), b, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
      why = cudaGetErrorString(e);
      return false;
    }
  }
  return true;
}

}  // namespace

extern "C" {

zoom_status zoom_dict_save(zoom_dict d, const char* path, void* stream) {
  if (!d || !path) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaSetDevice(d->ctx->device) != cudaSuccess) return fail(ZOOM_ERR_CUDA, "cudaSetDevice");
  File fl(path, "wb");
  if (!fl.f) return fail(ZOOM_ERR_IO, std::string("cannot open ") + path);
  DictHeader h{};
  memcpy(h.magic, kDictMagic, 8);
  h.version = kVersion;
  h.feature = (uint32_t)d->feature;
  h.n = d->n;
  h.P = d->P;
  h.s = d->s;
  h.d = d->d;
  h.dpad = d->dpad;
  h.ph2 = d->ph2;
  h.ph2pad = d->ph2pad;
  h.blur_sigma = d->blur_sigma;
  if (fwrite(&h, sizeof(h), 1, fl.f) != 1) return fail(ZOOM_ERR_IO, "write failed");
  std::vector<char> stage(kStage);
  std::string why;
  const int64_t n = d->n;
  if (!write_dev(fl.f, d->lr_pix, (size_t)n * d->P * d->P * 4, stage, st, why) ||
      !write_dev(fl.f, d->feat, (size_t)n * d->dpad * 4, stage, st, why) ||
      !write_dev(fl.f, d->mu, (size_t)n * 4, stage, st, why) ||
      !write_dev(fl.f, d->norm2, (size_t)n * 4, stage, st, why) ||
      !write_dev(fl.f, d->hr_res, (size_t)n * d->ph2pad * 4, stage, st, why))
    return fail(why == "write failed" ? ZOOM_ERR_IO : ZOOM_ERR_CUDA, "dictionary save: " + why);
  if (fflush(fl.f) != 0) return fail(ZOOM_ERR_IO, "write failed");
  return ZOOM_OK;
}

zoom_status zoom_dict_load(zoom_ctx ctx, const char* path, void* stream, zoom_dict* out) {
  if (!ctx || !path || !out) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  File fl(path, "rb");
  if (!fl.f) return fail(ZOOM_ERR_IO, std::string("cannot open ") + path);
  DictHeader h{};
  if (fread(&h, sizeof(h), 1, fl.f) != 1) return fail(ZOOM_ERR_IO, "file truncated");
  if (memcmp(h.magic, kDictMagic, 8) != 0) return fail(ZOOM_ERR_INVALID_ARG, "not a dictionary file");
  if (h.version != kVersion) return fail(ZOOM_ERR_INVALID_ARG, "unsupported dictionary file version");
  if ((h.P != 3 && h.P != 5) || h.s < 1 || h.s > 4 || h.n < 1 || h.n > (1LL << 30) || h.feature > 2 ||
      h.d != (h.feature ? 2 : 1) * h.P * h.P ||
      h.dpad != (h.d + 3) / 4 * 4 || h.ph2 != h.s * h.P * h.s * h.P || h.ph2pad != (h.ph2 + 3) / 4 * 4 ||
      !(h.blur_sigma > 0.0))
    return fail(ZOOM_ERR_INVALID_ARG, "dictionary file header out of range");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return fail(ZOOM_ERR_CUDA, "cudaSetDevice");
  zoom_dict d = zoom_dict_alloc(ctx, h.n, h.P, h.s, h.blur_sigma, (int)h.feature, st);
  if (!d) return fail(ZOOM_ERR_OOM, "dictionary arrays");
  std::vector<char> stage(kStage);
  std::string why;
  const int64_t n = d->n;
  const bool ok = read_dev(fl.f, d->lr_pix, (size_t)n * d->P * d->P * 4, stage, st, why) &&
                  read_dev(fl.f, d->feat, (size_t)n * d->dpad * 4, stage, st, why) &&
                  read_dev(fl.f, d->mu, (size_t)n * 4, stage, st, why) &&
                  read_dev(fl.f, d->norm2, (size_t)n * 4, stage, st, why) &&
                  read_dev(fl.f, d->hr_res, (size_t)n * d->ph2pad * 4, stage, st, why);
  if (!ok) {
    zoom_dict_destroy(d);
    return fail(why == "file truncated" ? ZOOM_ERR_IO : ZOOM_ERR_CUDA, "dictionary load: " + why);
  }
  *out = d;
  return ZOOM_OK;
}

zoom_status zoom_export_params(zoom_index ix, float* alpha, float* beta, void* stream) {
  if (!ix) return fail(ZOOM_ERR_INVALID_ARG, "NULL index");
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaSetDevice(ix->dict->ctx->device) != cudaSuccess) return fail(ZOOM_ERR_CUDA, "cudaSetDevice");
  const size_t na = (size_t)ix->L * ix->k * ix->dict->d, nb = (size_t)ix->L * ix->k;
  cudaError_t e = cudaSuccess;
  if (alpha) e = cudaMemcpyAsync(alpha, ix->alpha, na * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && beta) e = cudaMemcpyAsync(beta, ix->beta, nb * 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail(ZOOM_ERR_CUDA, std::string("export params: ") + cudaGetErrorString(e));
  return ZOOM_OK;
}

zoom_status zoom_index_save(zoom_index ix, const char* path, void* stream) {
  if (!ix || !path) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  const size_t na = (size_t)ix->L * ix->k * ix->dict->d, nb = (size_t)ix->L * ix->k;
  std::vector<float> alpha(na), beta(nb);
  zoom_status rc = zoom_export_params(ix, alpha.data(), beta.data(), stream);
  if (rc != ZOOM_OK) return rc;
  File fl(path, "wb");
  if (!fl.f) return fail(ZOOM_ERR_IO, std::string("cannot open ") + path);
  IndexHeader h{};
  memcpy(h.magic, kIndexMagic, 8);
  h.version = kVersion;
  h.n = ix->dict->n;
  h.d = ix->dict->d;
  h.L = ix->L;
  h.k = ix->k;
  h.t = ix->t;
  h.cap = ix->cap;
  h.w = ix->w;
  if (fwrite(&h, sizeof(h), 1, fl.f) != 1 || fwrite(alpha.data(), 4, na, fl.f) != na ||
      fwrite(beta.data(), 4, nb, fl.f) != nb || fflush(fl.f) != 0)
    return fail(ZOOM_ERR_IO, "write failed");
  return ZOOM_OK;
}

zoom_status zoom_index_load(zoom_dict d, const char* path, void* stream, zoom_index* out) {
  if (!d || !path || !out) return fail(ZOOM_ERR_INVALID_ARG, "NULL argument");
  File fl(path, "rb");
  if (!fl.f) return fail(ZOOM_ERR_IO, std::string("cannot open ") + path);
  IndexHeader h{};
  if (fread(&h, sizeof(h), 1, fl.f) != 1) return fail(ZOOM_ERR_IO, "file truncated");
  if (memcmp(h.magic, kIndexMagic, 8) != 0) return fail(ZOOM_ERR_INVALID_ARG, "not an index file");
  if (h.version != kVersion) return fail(ZOOM_ERR_INVALID_ARG, "unsupported index file version");
  if (h.n != d->n || h.d != d->d)
    return fail(ZOOM_ERR_INVALID_ARG, "index file does not belong to this dictionary");
  if (h.L < 1 || h.L > 32 || h.k < 1 || h.k > 32)
    return fail(ZOOM_ERR_INVALID_ARG, "index file header out of range");
  const size_t na = (size_t)h.L * h.k * h.d, nb = (size_t)h.L * h.k;
  std::vector<float> alpha(na), beta(nb);
  if (fread(alpha.data(), 4, na, fl.f) != na || fread(beta.data(), 4, nb, fl.f) != nb)
    return fail(ZOOM_ERR_IO, "file truncated");
  zoom_lsh_params p{};
  p.L = h.L;
  p.k = h.k;
  p.w = h.w;
  p.min_table_hits = h.t;
  p.max_candidates = h.cap;
  return zoom_build_index(d, &p, alpha.data(), beta.data(), stream, out);
}

}  // extern "C"
