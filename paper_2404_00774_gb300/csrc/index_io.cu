// Saving and loading a built index (the inverted lists of Section 2.2 with
// the spilled copies of Section 3.5, and every layout the search kernels
// read), so that a large index is built once.
//
// File format (little-endian, no padding between sections):
//   header   struct FileHeader below (magic "SOARIDX1", format version 2,
//            the scalar fields of the index, then the byte size of every
//            array section in the fixed order of kSections)
//   arrays   each present array's bytes, in that order
// An absent array (for example the FP8 scales of an fp32 index) has size 0.
// Arrays move through a pinned host buffer in chunks of kChunk bytes with one
// cudaMemcpyAsync per chunk on the caller's stream.
#include <sys/stat.h>

#include <cstdio>
#include <cstring>
#include <memory>

#include "internal.cuh"

namespace soar {

namespace {

constexpr char kMagic[8] = {'S', 'O', 'A', 'R', 'I', 'D', 'X', '1'};
constexpr uint32_t kVersion = 2;
constexpr int kSections = 17;
constexpr size_t kChunk = size_t(64) << 20;

struct FileHeader {
  char magic[8];
  uint32_t version;
  uint32_t header_bytes;
  int64_t n, rows, max_partition, tc_groups, bytes;
  int32_t d, c, spills, mode, dtype, row_stride, code_stride, tc_kp, sel_kp, sel_tiles, pq_m, reserved;
  uint64_t section_bytes[kSections];
};

// Device pointer of every array section with the byte size the index's
// scalar fields give it, in file order (an absent array: a null pointer).
struct Section {
  void** ptr;
  size_t bytes;
};

void sections(IndexData& ix, Section (&out)[kSections]) {
  const size_t esz = ix.dtype == SOAR_F32 ? 4 : 2;
  const bool coded = ix.mode == SOAR_SCORE_FP8 || ix.mode == SOAR_SCORE_PQ4;   // byte codes per copy
  const size_t vec_bytes = coded ? (size_t)ix.rows * ix.code_stride : esz * (size_t)ix.rows * ix.row_stride;
  const int ostride = (int)(((ix.d * esz + 15) / 16) * 16 / esz);
  int i = 0;
  auto add = [&](void** p, size_t b) { out[i++] = Section{p, b}; };
  add((void**)&ix.offsets, sizeof(int64_t) * (ix.c + 1));
  add((void**)&ix.ids, sizeof(int32_t) * ix.rows);
  add(&ix.vectors, vec_bytes);
  add((void**)&ix.row_scales, sizeof(float) * ix.rows);
  add(&ix.originals, esz * (size_t)ix.n * ostride);
  add((void**)&ix.centroids, sizeof(float) * (size_t)ix.c * ix.d);
  add((void**)&ix.part_order, sizeof(int32_t) * ix.c);
  add((void**)&ix.cent_code_vals, sizeof(float) * (size_t)ix.c * ix.code_stride);
  add((void**)&ix.cent_scales, sizeof(float) * ix.c);
  add(&ix.tc_rows, esz * (size_t)ix.tc_groups * 8 * ix.tc_kp);
  add((void**)&ix.tc_gstart, sizeof(int64_t) * (ix.c + 1));
  add((void**)&ix.tc_ids, sizeof(int32_t) * (size_t)ix.tc_groups * 8);
  add((void**)&ix.tc_norms, sizeof(float) * (size_t)ix.tc_groups * 8);
  add((void**)&ix.tc_pmax, sizeof(float) * ix.c);
  add((void**)&ix.assign, sizeof(int32_t) * (size_t)ix.n * (1 + ix.spills));
  add((void**)&ix.sel_cb, sizeof(float) * 2 * 64 * (size_t)ix.sel_kp * ix.sel_tiles);
  add((void**)&ix.pq_cb, sizeof(float) * (size_t)ix.pq_m * 16 * 2);
}

struct File {
  FILE* f = nullptr;
  ~File() {
    if (f) fclose(f);
  }
};

struct Pinned {
  void* p = nullptr;
  ~Pinned() {
    if (p) cudaFreeHost(p);
  }
};

}  // namespace

void save_index(const IndexData& ix_in, const char* path, cudaStream_t s) {
  IndexData ix = ix_in;   // shallow copy: only its pointers are read
  Section sec[kSections];
  sections(ix, sec);
  FileHeader h{};
  memcpy(h.magic, kMagic, 8);
  h.version = kVersion;
  h.header_bytes = sizeof(FileHeader);
  h.n = ix.n; h.rows = ix.rows; h.max_partition = ix.max_partition; h.tc_groups = ix.tc_groups; h.bytes = ix.bytes;
  h.d = ix.d; h.c = ix.c; h.spills = ix.spills; h.mode = ix.mode; h.dtype = ix.dtype; h.row_stride = ix.row_stride;
  h.code_stride = ix.code_stride; h.tc_kp = ix.tc_kp; h.sel_kp = ix.sel_kp; h.sel_tiles = ix.sel_tiles;
  h.pq_m = ix.pq_m;
  for (int i = 0; i < kSections; ++i) h.section_bytes[i] = *sec[i].ptr ? sec[i].bytes : 0;
  File f;
  f.f = fopen(path, "wb");
  if (!f.f) fail(SOAR_EINVAL, std::string("soar_index_save: cannot open ") + path + " for writing");
  if (fwrite(&h, sizeof(h), 1, f.f) != 1) fail(SOAR_ECUDA, "soar_index_save: write failed");
  Pinned buf;
  SOAR_CUDA(cudaMallocHost(&buf.p, kChunk));
  for (int i = 0; i < kSections; ++i) {
    const char* src = static_cast<const char*>(*sec[i].ptr);
    for (size_t off = 0; off < h.section_bytes[i]; off += kChunk) {
      const size_t b = std::min(kChunk, (size_t)h.section_bytes[i] - off);
      SOAR_CUDA(cudaMemcpyAsync(buf.p, src + off, b, cudaMemcpyDeviceToHost, s));
      SOAR_CUDA(cudaStreamSynchronize(s));
      if (fwrite(buf.p, 1, b, f.f) != b) fail(SOAR_ECUDA, "soar_index_save: write failed (disk full?)");
    }
  }
  if (fflush(f.f) != 0) fail(SOAR_ECUDA, "soar_index_save: flush failed");
}

void load_index(IndexData& ix, const char* path, cudaStream_t s) {
  File f;
  f.f = fopen(path, "rb");
  if (!f.f) fail(SOAR_EINVAL, std::string("soar_index_load: cannot open ") + path);
  FileHeader h{};
  if (fread(&h, sizeof(h), 1, f.f) != 1 || memcmp(h.magic, kMagic, 8) != 0)
    fail(SOAR_EINVAL, "soar_index_load: not a SOAR index file");
  if (h.version != kVersion || h.header_bytes != sizeof(FileHeader))
    fail(SOAR_EUNSUPPORTED, "soar_index_load: unsupported format version");
  const bool sane = h.n >= 1 && h.d >= 1 && h.d <= 4096 && h.c >= 1 && h.spills >= 0 && h.spills <= 4 &&
                    h.rows == h.n * (1 + h.spills) &&
                    (h.mode == SOAR_SCORE_F32 || h.mode == SOAR_SCORE_FP8 || h.mode == SOAR_SCORE_PQ4) &&
                    (h.mode == SOAR_SCORE_PQ4 ? h.pq_m == h.d / 2 : h.pq_m == 0) &&
                    (h.dtype == SOAR_F32 || h.dtype == SOAR_BF16);
  if (!sane) fail(SOAR_EINVAL, "soar_index_load: header fields out of range");
  ix.n = h.n; ix.rows = h.rows; ix.max_partition = h.max_partition; ix.tc_groups = h.tc_groups;
  ix.d = h.d; ix.c = h.c; ix.spills = h.spills; ix.mode = h.mode; ix.dtype = h.dtype; ix.row_stride = h.row_stride;
  ix.code_stride = h.code_stride; ix.tc_kp = h.tc_kp; ix.sel_kp = h.sel_kp; ix.sel_tiles = h.sel_tiles;
  ix.pq_m = h.pq_m;
  // every section the file carries must have the size the header's fields
  // give it; the offsets, ids, vectors and centroids must be present
  Section sec[kSections];
  sections(ix, sec);
  for (int i = 0; i < kSections; ++i) {
    if (h.section_bytes[i] != 0 && h.section_bytes[i] != sec[i].bytes)
      fail(SOAR_EINVAL, "soar_index_load: section " + std::to_string(i) + " has the wrong size");
    if (h.section_bytes[i] == 0 && (i == 0 || i == 1 || i == 2 || i == 5 || (i == 16 && h.mode == SOAR_SCORE_PQ4)))
      fail(SOAR_EINVAL, "soar_index_load: a required section is missing");
  }
  // the file holds exactly the header and the sections it lists, checked on
  // the host before any device memory is taken (the reads below check again)
  uint64_t want = sizeof(FileHeader);
  for (int i = 0; i < kSections; ++i) want += h.section_bytes[i];
  struct stat st;
  if (stat(path, &st) != 0) fail(SOAR_EINVAL, std::string("soar_index_load: cannot stat ") + path);
  if ((uint64_t)st.st_size < want) fail(SOAR_EINVAL, "soar_index_load: file is truncated");
  if ((uint64_t)st.st_size > want) fail(SOAR_EINVAL, "soar_index_load: trailing bytes after the last section");
  for (int i = 0; i < kSections; ++i) {
    if (h.section_bytes[i] == 0) continue;
    SOAR_CUDA(cudaMalloc(sec[i].ptr, sec[i].bytes));
    ix.bytes += (int64_t)sec[i].bytes;
  }
  Pinned buf;
  SOAR_CUDA(cudaMallocHost(&buf.p, kChunk));
  for (int i = 0; i < kSections; ++i) {
    char* dst = static_cast<char*>(*sec[i].ptr);
    for (size_t off = 0; off < h.section_bytes[i]; off += kChunk) {
      const size_t b = std::min(kChunk, (size_t)h.section_bytes[i] - off);
      if (fread(buf.p, 1, b, f.f) != b) fail(SOAR_EINVAL, "soar_index_load: file is truncated");
      SOAR_CUDA(cudaMemcpyAsync(dst + off, buf.p, b, cudaMemcpyHostToDevice, s));
      SOAR_CUDA(cudaStreamSynchronize(s));
    }
  }
  char extra;
  if (fread(&extra, 1, 1, f.f) != 0) fail(SOAR_EINVAL, "soar_index_load: trailing bytes after the last section");
}

}  // namespace soar
