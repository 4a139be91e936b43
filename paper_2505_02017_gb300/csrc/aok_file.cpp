// Chunk-blob files: the on-disk form of a scene's (chunk, LOD) blobs (the
// paper streams preprocessed chunks from disk, Sec. 3.4; Table 1 "Disk").
// A file is written once (aok_blobfile_create / _add / _finish) and read by
// any number of threads (aok_blobfile_open, aok_blobfile_read); the reader is
// also a chunk source for aok_stream.
//
// Layout (little-endian):
//   header  64 B  magic "AOKBLOB1", version, chunk_res, n_lods, grid[3],
//                 n_entries, index offset, index checksum, header checksum
//   entries       per (chunk, LOD), 8-byte aligned: a 56-byte entry header
//                 (word counts, root, AABB), nodes, padding to 8 bytes,
//                 leaves, colours
//   index         n_entries x {chunk, lod, offset, size, checksum}, sorted by
//                 (chunk, lod)
// Checksums are 64-bit FNV-1a over the bytes they cover; a reader rejects a
// file whose header or index does not check, and a read whose entry does not.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <fcntl.h>
#include <sys/stat.h>
#include <unistd.h>

#include "aok.h"

namespace {

constexpr char kMagic[8] = {'A', 'O', 'K', 'B', 'L', 'O', 'B', '1'};
constexpr uint32_t kVersion = 1;

uint64_t fnv1a(const void* p, size_t n, uint64_t h = 0xcbf29ce484222325ull) {
    const uint8_t* b = (const uint8_t*)p;
    for (size_t i = 0; i < n; i++) {
        h ^= b[i];
        h *= 0x100000001b3ull;
    }
    return h;
}

struct FileHeader {
    char magic[8];
    uint32_t version, chunk_res, n_lods, grid[3];
    uint64_t n_entries, index_offset, index_sum, header_sum;  // header_sum over the bytes before it
};
static_assert(sizeof(FileHeader) == 64, "64-byte header");

struct EntryHeader {
    uint64_t n_node_words, n_leaves, n_mats;
    uint32_t root;
    int32_t aabb_lo[3], aabb_hi[3];
    uint32_t pad;
};
static_assert(sizeof(EntryHeader) == 56, "entry header");

struct IndexEntry {
    uint64_t chunk;
    uint32_t lod, pad;
    uint64_t offset, size, sum;
};

// entry body: [EntryHeader][nodes][pad to 8][leaves][colours]
uint64_t leaves_offset(uint64_t n_node_words) { return (sizeof(EntryHeader) + n_node_words * 4 + 7) & ~7ull; }

bool write_all(int fd, const void* p, size_t n) {
    const char* c = (const char*)p;
    while (n) {
        const ssize_t w = ::write(fd, c, n);
        if (w <= 0) return false;
        c += w;
        n -= (size_t)w;
    }
    return true;
}

bool pread_all(int fd, void* p, size_t n, uint64_t off) {
    char* c = (char*)p;
    while (n) {
        const ssize_t r = ::pread(fd, c, n, (off_t)off);
        if (r <= 0) return false;
        c += r;
        n -= (size_t)r;
        off += (uint64_t)r;
    }
    return true;
}

}  // namespace

struct aok_blobfile {
    int fd = -1;
    bool writing = false;
    FileHeader hdr{};
    std::vector<IndexEntry> index;
    uint64_t end = 0;  // writing: next entry offset
    std::mutex mu;     // writing: one add at a time
};

extern "C" {

int aok_blobfile_create(const char* path, int32_t chunk_res, int32_t n_lods, const int32_t grid[3],
                        aok_blobfile** out) {
    if (!path || !out || chunk_res < 8 || n_lods < 1 || n_lods > 8 || !grid || grid[0] < 1 || grid[1] < 1 ||
        grid[2] < 1)
        return AOK_E_INVALID;
    const int fd = ::open(path, O_CREAT | O_TRUNC | O_WRONLY, 0644);
    if (fd < 0) return AOK_E_INVALID;
    aok_blobfile* f = new (std::nothrow) aok_blobfile();
    if (!f) {
        ::close(fd);
        return AOK_E_OOM;
    }
    f->fd = fd;
    f->writing = true;
    std::memcpy(f->hdr.magic, kMagic, 8);
    f->hdr.version = kVersion;
    f->hdr.chunk_res = (uint32_t)chunk_res;
    f->hdr.n_lods = (uint32_t)n_lods;
    for (int a = 0; a < 3; a++) f->hdr.grid[a] = (uint32_t)grid[a];
    f->end = sizeof(FileHeader);
    // placeholder header, rewritten by aok_blobfile_finish
    if (!write_all(fd, &f->hdr, sizeof(FileHeader))) {
        ::close(fd);
        delete f;
        return AOK_E_INVALID;
    }
    *out = f;
    return AOK_OK;
}

int aok_blobfile_add(aok_blobfile* f, int64_t chunk, uint32_t lod, const aok_chunk_blob* b) {
    if (!f || !f->writing || !b || chunk < 0 || lod >= f->hdr.n_lods) return AOK_E_INVALID;
    const uint64_t n_chunks = (uint64_t)f->hdr.grid[0] * f->hdr.grid[1] * f->hdr.grid[2];
    if ((uint64_t)chunk >= n_chunks) return AOK_E_INVALID;
    EntryHeader eh{};
    eh.n_node_words = b->n_node_words;
    eh.n_leaves = b->n_leaves;
    eh.n_mats = b->n_mats;
    eh.root = b->root;
    for (int a = 0; a < 3; a++) { eh.aabb_lo[a] = b->aabb_lo[a]; eh.aabb_hi[a] = b->aabb_hi[a]; }
    const uint64_t leaf_at = leaves_offset(eh.n_node_words);
    const uint64_t body = leaf_at + eh.n_leaves * 8 + eh.n_mats;
    const uint64_t padded = (body + 7) & ~7ull;
    std::vector<char> buf(padded, 0);
    std::memcpy(buf.data(), &eh, sizeof(eh));
    if (eh.n_node_words) std::memcpy(buf.data() + sizeof(eh), b->nodes, eh.n_node_words * 4);
    if (eh.n_leaves) std::memcpy(buf.data() + leaf_at, b->leaves, eh.n_leaves * 8);
    if (eh.n_mats) std::memcpy(buf.data() + leaf_at + eh.n_leaves * 8, b->mats, eh.n_mats);
    std::lock_guard<std::mutex> g(f->mu);
    for (const IndexEntry& e : f->index)
        if (e.chunk == (uint64_t)chunk && e.lod == lod) return AOK_E_INVALID;  // one blob per (chunk, LOD)
    if (!write_all(f->fd, buf.data(), padded)) return AOK_E_INVALID;
    f->index.push_back({(uint64_t)chunk, lod, 0, f->end, padded, fnv1a(buf.data(), padded)});
    f->end += padded;
    return AOK_OK;
}

int aok_blobfile_finish(aok_blobfile* f) {
    if (!f || !f->writing) return AOK_E_INVALID;
    std::sort(f->index.begin(), f->index.end(), [](const IndexEntry& a, const IndexEntry& b) {
        return a.chunk != b.chunk ? a.chunk < b.chunk : a.lod < b.lod;
    });
    const size_t ib = f->index.size() * sizeof(IndexEntry);
    bool ok = f->index.empty() || write_all(f->fd, f->index.data(), ib);
    f->hdr.n_entries = f->index.size();
    f->hdr.index_offset = f->end;
    f->hdr.index_sum = fnv1a(f->index.data(), ib);
    f->hdr.header_sum = fnv1a(&f->hdr, offsetof(FileHeader, header_sum));
    ok = ok && ::pwrite(f->fd, &f->hdr, sizeof(FileHeader), 0) == (ssize_t)sizeof(FileHeader);
    ok = (::fsync(f->fd) == 0) && ok;
    ::close(f->fd);
    delete f;
    return ok ? AOK_OK : AOK_E_INVALID;
}

int aok_blobfile_open(const char* path, aok_blobfile** out) {
    if (!path || !out) return AOK_E_INVALID;
    const int fd = ::open(path, O_RDONLY);
    if (fd < 0) return AOK_E_INVALID;
    struct stat stt;
    FileHeader h;
    if (::fstat(fd, &stt) != 0 || !pread_all(fd, &h, sizeof(h), 0) || std::memcmp(h.magic, kMagic, 8) != 0 ||
        h.version != kVersion || h.header_sum != fnv1a(&h, offsetof(FileHeader, header_sum)) ||
        h.n_entries > (uint64_t)stt.st_size / sizeof(IndexEntry) || h.index_offset > (uint64_t)stt.st_size ||
        h.index_offset + h.n_entries * sizeof(IndexEntry) != (uint64_t)stt.st_size) {
        ::close(fd);
        return AOK_E_CORRUPT;
    }
    aok_blobfile* f = new (std::nothrow) aok_blobfile();
    if (!f) {
        ::close(fd);
        return AOK_E_OOM;
    }
    f->fd = fd;
    f->hdr = h;
    f->index.resize(h.n_entries);
    if ((h.n_entries && !pread_all(fd, f->index.data(), h.n_entries * sizeof(IndexEntry), h.index_offset)) ||
        fnv1a(f->index.data(), h.n_entries * sizeof(IndexEntry)) != h.index_sum) {
        ::close(fd);
        delete f;
        return AOK_E_CORRUPT;
    }
    for (const IndexEntry& e : f->index)
        if (e.offset < sizeof(FileHeader) || e.offset + e.size > h.index_offset || e.size < sizeof(EntryHeader)) {
            ::close(fd);
            delete f;
            return AOK_E_CORRUPT;
        }
    *out = f;
    return AOK_OK;
}

int aok_blobfile_info(const aok_blobfile* f, int32_t* chunk_res, int32_t* n_lods, int32_t grid[3],
                      uint64_t* n_entries) {
    if (!f) return AOK_E_INVALID;
    if (chunk_res) *chunk_res = (int32_t)f->hdr.chunk_res;
    if (n_lods) *n_lods = (int32_t)f->hdr.n_lods;
    if (grid) for (int a = 0; a < 3; a++) grid[a] = (int32_t)f->hdr.grid[a];
    if (n_entries) *n_entries = f->writing ? f->index.size() : f->hdr.n_entries;
    return AOK_OK;
}

int aok_blobfile_read(aok_blobfile* f, int64_t chunk, uint32_t lod, aok_chunk_blob* out, void** handle) {
    if (!f || f->writing || !out || !handle) return AOK_E_INVALID;
    *handle = nullptr;
    const IndexEntry key{(uint64_t)chunk, lod, 0, 0, 0, 0};
    auto it = std::lower_bound(f->index.begin(), f->index.end(), key, [](const IndexEntry& a, const IndexEntry& b) {
        return a.chunk != b.chunk ? a.chunk < b.chunk : a.lod < b.lod;
    });
    if (it == f->index.end() || it->chunk != (uint64_t)chunk || it->lod != lod) return AOK_E_NOT_RESIDENT;
    char* buf = new (std::nothrow) char[it->size];
    if (!buf) return AOK_E_OOM;
    if (!pread_all(f->fd, buf, it->size, it->offset) || fnv1a(buf, it->size) != it->sum) {
        delete[] buf;
        return AOK_E_CORRUPT;
    }
    EntryHeader eh;
    std::memcpy(&eh, buf, sizeof(eh));
    const uint64_t leaf_at = leaves_offset(eh.n_node_words);
    if (eh.n_node_words > it->size || eh.n_leaves > it->size || eh.n_mats > it->size ||
        leaf_at + eh.n_leaves * 8 + eh.n_mats > it->size) {
        delete[] buf;
        return AOK_E_CORRUPT;
    }
    out->nodes = (const uint32_t*)(buf + sizeof(EntryHeader));
    out->n_node_words = eh.n_node_words;
    out->leaves = (const uint64_t*)(buf + leaf_at);
    out->n_leaves = eh.n_leaves;
    out->mats = (const uint8_t*)(buf + leaf_at + eh.n_leaves * 8);
    out->n_mats = eh.n_mats;
    out->root = eh.root;
    for (int a = 0; a < 3; a++) { out->aabb_lo[a] = eh.aabb_lo[a]; out->aabb_hi[a] = eh.aabb_hi[a]; }
    *handle = buf;
    return AOK_OK;
}

void aok_blobfile_release(void* user, void* handle) {
    (void)user;
    delete[] (char*)handle;
}

int aok_blobfile_source(void* user, int32_t cx, int32_t cy, int32_t cz, uint32_t lod, aok_chunk_blob* out,
                        void** handle) {
    aok_blobfile* f = (aok_blobfile*)user;
    if (!f || cx < 0 || cy < 0 || cz < 0 || (uint32_t)cx >= f->hdr.grid[0] || (uint32_t)cy >= f->hdr.grid[1] ||
        (uint32_t)cz >= f->hdr.grid[2])
        return AOK_E_INVALID;
    const int64_t chunk = (int64_t)cx + (int64_t)f->hdr.grid[0] * ((int64_t)cy + (int64_t)f->hdr.grid[1] * cz);
    const int st = aok_blobfile_read(f, chunk, lod, out, handle);
    if (st == AOK_E_NOT_RESIDENT) {
        // a (chunk, LOD) the file does not hold is an empty chunk
        std::memset(out, 0, sizeof(*out));
        *handle = nullptr;
        return 0;
    }
    return st == AOK_OK ? 0 : -1;
}

int aok_blobfile_close(aok_blobfile* f) {
    if (!f) return AOK_E_INVALID;
    if (f->writing) return aok_blobfile_finish(f);
    ::close(f->fd);
    delete f;
    return AOK_OK;
}

}  // extern "C"
