// On-disk storage of converted matrices (the paper's future work, Section 8: keep the formats
// so that a later run skips the conversion).  spmv_save writes the handle's CRS arrays and,
// when built, the Hilbert-ordered blocked arrays and the staged blocked layout; spmv_load
// restores them into a new handle whose conversions to those formats then cost only the cheap
// derived tables (merge partition, row bins, the HB chunk table, the CTA split of the staged
// layout for the loading device, the Merge Blocking block-row pointer and lane split points).
//
// File layout (host byte order; every array as stored on the device, without padding):
//   8-byte magic "SPMVGB01", uint32 version, uint32 section flags (1 CRS, 2 HB, 4 staged),
//   int64 m, n, nnz, int32 dtype, int32 active format, int32 hb_chunked, int32 reserved;
//   CRS: row_ptr (m+1 int32), col (nnz int32), values (nnz x element size);
//   HB: int32 log2beta, grid K, inner order, block order; int64 nblk; packed indices (nnz uint32),
//       values, blk_ptr (nblk+1), blk_row (nblk), blk_col (nblk) (int32);
//   staged: int32 lb, kind; int64 slices, tiles; tile headers (16 B each), words (256 x 4 B per
//       tile), values (256 per tile), first tile per slice (slices+1 uint32), lane headers
//       (256 B per tile).
#include "common.cuh"
#include "convert.cuh"

#include <cstdio>
#include <cstring>
#include <vector>

namespace spmv {
namespace {

constexpr char MAGIC[8] = {'S', 'P', 'M', 'V', 'G', 'B', '0', '1'};
constexpr uint32_t VERSION = 2;   // 2: lane headers carry the scan segment start, tile headers the scan levels
constexpr size_t CHUNK = 64u << 20;   // host staging per copy
constexpr size_t TMA_PAD = 64;        // the padding the conversion gives the CRS arrays

int stage_value_bytes(int32_t kind) { return kind == 1 || kind == 2 ? 8 : kind == 3 ? 4 : kind == 4 ? 2 : 0; }

struct File {
    FILE *f = nullptr;
    ~File() {
        if (f) fclose(f);
    }
};

spmv_status io_error(const char *what, const char *path) {
    set_error(std::string(what) + ": " + path);
    return SPMV_ERR_IO;
}

// Checksum of every array byte of the file (a word-wise multiply-xorshift hash), written at
// the end: a damaged or truncated file is rejected before any kernel reads what it holds.
struct Hash {
    uint64_t h = 0x243F6A8885A308D3ull;
    void add(const void *p, size_t n) {
        const unsigned char *b = (const unsigned char *)p;
        size_t i = 0;
        for (; i + 8 <= n; i += 8) {
            uint64_t w;
            memcpy(&w, b + i, 8);
            h = (h ^ w) * 0x9E3779B97F4A7C15ull;
            h ^= h >> 29;
        }
        uint64_t w = 0;
        memcpy(&w, b + i, n - i);
        h = (h ^ w ^ ((uint64_t)(n - i) << 56)) * 0x9E3779B97F4A7C15ull;
        h ^= h >> 29;
    }
};

// Device array -> file, through a pinned host buffer.
spmv_status put(FILE *f, const void *dev, size_t bytes, void *stage, cudaStream_t s, const char *path, Hash &hs) {
    for (size_t off = 0; off < bytes; off += CHUNK) {
        const size_t b = std::min(CHUNK, bytes - off);
        SPMV_CUDA_TRY(cudaMemcpyAsync(stage, (const char *)dev + off, b, cudaMemcpyDeviceToHost, s));
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));
        hs.add(stage, b);
        if (fwrite(stage, 1, b, f) != b) return io_error("spmv_save: write failed", path);
    }
    return SPMV_OK;
}

// File -> newly allocated device array of `bytes` (+ pad).
spmv_status get(FILE *f, void **dev, size_t bytes, size_t pad, void *stage, cudaStream_t s, const char *what,
                const char *path, Hash &hs) {
    DevBuf d(s);
    SPMV_TRY(d.alloc(bytes + pad, what));
    for (size_t off = 0; off < bytes; off += CHUNK) {
        const size_t b = std::min(CHUNK, bytes - off);
        SPMV_CUDA_TRY(cudaStreamSynchronize(s));   // the staging buffer is free again
        if (fread(stage, 1, b, f) != b) return io_error("spmv_load: file truncated", path);
        hs.add(stage, b);
        SPMV_CUDA_TRY(cudaMemcpyAsync((char *)d.p + off, stage, b, cudaMemcpyHostToDevice, s));
    }
    SPMV_CUDA_TRY(cudaStreamSynchronize(s));
    *dev = d.release();
    return SPMV_OK;
}

template <typename T>
bool wr(FILE *f, const T &v) { return fwrite(&v, sizeof v, 1, f) == 1; }
template <typename T>
bool rd(FILE *f, T &v) { return fread(&v, sizeof v, 1, f) == 1; }

struct Pinned {
    void *p = nullptr;
    ~Pinned() {
        if (p) cudaFreeHost(p);
    }
};

}  // namespace
}  // namespace spmv

using namespace spmv;

extern "C" {

spmv_status spmv_save(spmv_handle h, const char *path, void *stream) {
    if (!h || !path) {
        set_error("spmv_save: NULL handle or path");
        return SPMV_ERR_INVALID_ARG;
    }
    if (!h->has_csr) {
        set_error("spmv_save: the handle has no converted format (call spmv_convert first)");
        return SPMV_ERR_NOT_CONVERTED;
    }
    cudaStream_t s = (cudaStream_t)stream;
    File fl;
    if (!(fl.f = fopen(path, "wb"))) return io_error("spmv_save: cannot open", path);
    FILE *f = fl.f;
    Pinned stage;
    SPMV_CUDA_TRY(cudaMallocHost(&stage.p, CHUNK));
    Hash hs;
    const int es = elem_size(h->dt);
    const uint32_t sections = 1u | (h->has_hb ? 2u : 0u) | (h->has_stage ? 4u : 0u);
    const int32_t reserved = 0, hbc = h->hb_chunked ? 1 : 0;
    const int32_t dt = (int32_t)h->dt, fmt = h->format;
    bool ok = fwrite(MAGIC, 1, 8, f) == 8 && wr(f, VERSION) && wr(f, sections) && wr(f, h->m) && wr(f, h->n) &&
              wr(f, h->nnz) && wr(f, dt) && wr(f, fmt) && wr(f, hbc) && wr(f, reserved);
    if (!ok) return io_error("spmv_save: write failed", path);
    SPMV_TRY(put(f, h->row_ptr, (size_t)(h->m + 1) * 4, stage.p, s, path, hs));
    SPMV_TRY(put(f, h->col, (size_t)h->nnz * 4, stage.p, s, path, hs));
    if (es) SPMV_TRY(put(f, h->val, (size_t)h->nnz * es, stage.p, s, path, hs));
    if (h->has_hb) {
        ok = wr(f, h->log2beta) && wr(f, h->grid_K) && wr(f, h->inner) && wr(f, h->block_order) && wr(f, h->nblk);
        if (!ok) return io_error("spmv_save: write failed", path);
        SPMV_TRY(put(f, h->hb_idx, (size_t)h->nnz * 4, stage.p, s, path, hs));
        if (es) SPMV_TRY(put(f, h->hb_val, (size_t)h->nnz * es, stage.p, s, path, hs));
        SPMV_TRY(put(f, h->blk_ptr, (size_t)(h->nblk + 1) * 4, stage.p, s, path, hs));
        SPMV_TRY(put(f, h->blk_row, (size_t)h->nblk * 4, stage.p, s, path, hs));
        SPMV_TRY(put(f, h->blk_col, (size_t)h->nblk * 4, stage.p, s, path, hs));
    }
    if (h->has_stage) {
        ok = wr(f, h->stage_lb) && wr(f, h->stage_kind) && wr(f, h->stage_nsl) && wr(f, h->stage_tiles);
        if (!ok) return io_error("spmv_save: write failed", path);
        const size_t T = (size_t)h->stage_tiles;
        const int vs = stage_value_bytes(h->stage_kind);
        if (T) {
            SPMV_TRY(put(f, h->st_hdr, T * 16, stage.p, s, path, hs));
            SPMV_TRY(put(f, h->st_words, T * 256 * 4, stage.p, s, path, hs));
            if (vs) SPMV_TRY(put(f, h->st_vals, T * 256 * vs, stage.p, s, path, hs));
            SPMV_TRY(put(f, h->st_slice_tile, (size_t)(h->stage_nsl + 1) * 4, stage.p, s, path, hs));
            SPMV_TRY(put(f, h->st_lmeta, T * 256, stage.p, s, path, hs));
        }
    }
    if (!wr(f, hs.h) || fflush(f) != 0) return io_error("spmv_save: write failed", path);
    return SPMV_OK;
}

spmv_status spmv_load(const char *path, void *stream, spmv_handle *out) {
    if (!path || !out) {
        set_error("spmv_load: NULL path or output");
        return SPMV_ERR_INVALID_ARG;
    }
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    File fl;
    if (!(fl.f = fopen(path, "rb"))) return io_error("spmv_load: cannot open", path);
    FILE *f = fl.f;
    char magic[8];
    uint32_t version = 0, sections = 0;
    int64_t m = 0, n = 0, nnz = 0;
    int32_t dt = 0, fmt = 0, hbc = 0, reserved = 0;
    bool ok = fread(magic, 1, 8, f) == 8 && rd(f, version) && rd(f, sections) && rd(f, m) && rd(f, n) && rd(f, nnz) &&
              rd(f, dt) && rd(f, fmt) && rd(f, hbc) && rd(f, reserved);
    if (!ok || memcmp(magic, MAGIC, 8) != 0 || version != VERSION || !(sections & 1u) || m < 0 || n < 0 || nnz < 0 ||
        m >= ((int64_t)1 << 31) || n >= ((int64_t)1 << 31) || nnz >= ((int64_t)1 << 31) || dt < 0 || dt > 3 ||
        fmt < -1 || (fmt > 2 && fmt != SPMV_FMT_MERGEB)) {
        set_error(std::string("spmv_load: not a matrix file of this library, of another file format version, or a "
                              "damaged header: ") + path);
        return SPMV_ERR_INVALID_ARG;
    }
    // a handle with no triplets, then the stored arrays
    spmv_handle h = nullptr;
    SPMV_TRY(spmv_create_coo(m, n, 0, nullptr, nullptr, nullptr, (spmv_dtype)dt, 0, stream, &h));
    struct Guard {
        spmv_handle h;
        ~Guard() {
            if (h) spmv_destroy(h);
        }
    } guard{h};
    Pinned stage;
    SPMV_CUDA_TRY(cudaMallocHost(&stage.p, CHUNK));
    Hash hs;
    const int es = elem_size((spmv_dtype)dt);
    h->nnz = nnz;
    h->nnz_in = nnz;
    void *p = nullptr;
    SPMV_TRY(get(f, &p, (size_t)(m + 1) * 4, TMA_PAD, stage.p, s, "row_ptr", path, hs));
    h->row_ptr = (int32_t *)p;
    SPMV_TRY(get(f, &p, (size_t)nnz * 4, TMA_PAD, stage.p, s, "col_ind", path, hs));
    h->col = (int32_t *)p;
    if (es) {
        SPMV_TRY(get(f, &p, (size_t)nnz * es, TMA_PAD, stage.p, s, "values", path, hs));
        h->val = p;
    }
    h->has_csr = true;
    h->bytes = (m + 1) * 4 + nnz * (4 + es);
    if (sections & 2u) {
        int32_t lb = 0, K = 0, inner = 0, r2 = 0;
        int64_t nblk = 0;
        if (!(rd(f, lb) && rd(f, K) && rd(f, inner) && rd(f, r2) && rd(f, nblk)) || nblk < 0 || nblk > nnz ||
            lb < 1 || lb > 16 || inner < 0 || inner > 2 || r2 < 0 || r2 > 1)
            return io_error("spmv_load: damaged blocked section", path);
        SPMV_TRY(get(f, &p, (size_t)nnz * 4, 0, stage.p, s, "hb idx", path, hs));
        h->hb_idx = (uint32_t *)p;
        if (es) {
            SPMV_TRY(get(f, &p, (size_t)nnz * es, 0, stage.p, s, "hb values", path, hs));
            h->hb_val = p;
        }
        SPMV_TRY(get(f, &p, (size_t)(nblk + 1) * 4, 0, stage.p, s, "hb blk_ptr", path, hs));
        h->blk_ptr = (int32_t *)p;
        SPMV_TRY(get(f, &p, (size_t)nblk * 4, 0, stage.p, s, "hb blk_row", path, hs));
        h->blk_row = (int32_t *)p;
        SPMV_TRY(get(f, &p, (size_t)nblk * 4, 0, stage.p, s, "hb blk_col", path, hs));
        h->blk_col = (int32_t *)p;
        h->nblk = nblk;
        h->log2beta = lb;
        h->grid_K = K;
        h->inner = inner;
        h->block_order = r2;
        h->has_hb = true;
        h->bytes += nnz * (4 + es) + nblk * 12 + 4;
    }
    SPMV_TRY(build_df(h, s));   // the double-float window of the values (as a conversion would)
    if (sections & 4u) {
        int32_t lb = 0, kind = 0;
        int64_t nsl = 0, T = 0;
        if (!(rd(f, lb) && rd(f, kind) && rd(f, nsl) && rd(f, T)) || lb < 1 || lb > 16 || nsl < 0 || T < 0 ||
            kind < 0 || kind > 4 || (kind == 1 && !h->df_ok))
            return io_error("spmv_load: damaged staged section", path);
        const int vs = stage_value_bytes(kind);
        if (T) {
            SPMV_TRY(get(f, &p, (size_t)T * 16, 0, stage.p, s, "stage tile headers", path, hs));
            h->st_hdr = (int4 *)p;
            SPMV_TRY(get(f, &p, (size_t)T * 256 * 4, 0, stage.p, s, "stage words", path, hs));
            h->st_words = (uint32_t *)p;
            if (vs) {
                SPMV_TRY(get(f, &p, (size_t)T * 256 * vs, 0, stage.p, s, "stage values", path, hs));
                h->st_vals = p;
            }
            SPMV_TRY(get(f, &p, (size_t)(nsl + 1) * 4, 0, stage.p, s, "stage slice tiles", path, hs));
            h->st_slice_tile = (uint32_t *)p;
            SPMV_TRY(get(f, &p, (size_t)T * 256, 0, stage.p, s, "stage lane headers", path, hs));
            h->st_lmeta = (uint2 *)p;
        }
        h->stage_lb = lb;
        h->stage_kind = kind;
        h->stage_nsl = nsl;
        h->stage_tiles = T;
        h->stage_bytes = T * (16 + 256 + 256 * (4 + (int64_t)vs)) + (nsl + 1) * 4;
        h->bytes += h->stage_bytes;
        h->has_stage = true;
    }
    uint64_t stored = 0;
    if (!rd(f, stored) || stored != hs.h) return io_error("spmv_load: checksum mismatch (damaged file)", path);
    // derived tables, from arrays now known to be the ones saved
    if (h->has_hb) SPMV_TRY(hb_chunk_table(h, s));
    if (h->has_stage) SPMV_TRY(stage_resplit(h, s));
    h->hb_chunked = hbc != 0;
    // the active format: its derived tables are cheap to rebuild from the stored arrays
    if (fmt >= 0) {
        spmv_convert_opts o = {h->has_hb ? h->log2beta : 0, h->has_hb ? h->inner : 0, 0,
                               hbc ? SPMV_HB_CHUNKED : SPMV_HB_STAGED, h->has_hb ? h->block_order : 0};
        SPMV_TRY(spmv_convert(h, (spmv_format)fmt, &o, stream));
    }
    guard.h = nullptr;
    *out = h;
    return SPMV_OK;
}

}  // extern "C"
