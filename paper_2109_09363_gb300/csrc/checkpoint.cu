// Network checkpoint files: the parameters of a network (FP32 masters) and,
// from a trainer, its Adam moments and step count (the paper trains its
// networks with a gradient-descent algorithm, Sec. 3.2; a run that stops
// resumes from such a file).  Host code only.
//
// Layout (little-endian, both hosts this library builds for are):
//   char     magic[8]   "HPCNNCK1"
//   uint32   version    1
//   int32    arch       hp_cnn_arch
//   int64    n          parameter count of that architecture
//   int64    step       Adam steps taken (0 for a network saved alone)
//   uint32   moments    1 when the Adam moments follow the parameters
//   uint32   reserved   0
//   float32  w[n]       parameters in network order (as hp_cnn_set_params)
//   float32  m[n], v[n] first and second Adam moments (moments == 1)
//   uint64   checksum   FNV-1a (64 bit) of every byte before it
#include <stdint.h>
#include <stdio.h>
#include <string.h>
#include <sys/types.h>

#include <string>
#include <vector>

#include "hproj_internal.cuh"

namespace hp {

namespace {

constexpr char kMagic[8] = {'H', 'P', 'C', 'N', 'N', 'C', 'K', '1'};
constexpr uint32_t kVersion = 1;

struct Header {
    char magic[8];
    uint32_t version;
    int32_t arch;
    int64_t n;
    int64_t step;
    uint32_t moments;
    uint32_t reserved;
};
static_assert(sizeof(Header) == 40, "checkpoint header is 40 bytes");

struct Fnv {
    uint64_t h = 1469598103934665603ull;
    void add(const void* p, size_t n)
    {
        const unsigned char* b = (const unsigned char*)p;
        for (size_t i = 0; i < n; ++i) {
            h ^= b[i];
            h *= 1099511628211ull;
        }
    }
};

bool put(FILE* f, Fnv& fnv, const void* p, size_t n)
{
    fnv.add(p, n);
    return fwrite(p, 1, n, f) == n;
}

bool get(FILE* f, Fnv& fnv, void* p, size_t n)
{
    if (fread(p, 1, n, f) != n) return false;
    fnv.add(p, n);
    return true;
}

}  // namespace

hp_status ckpt_write(const char* path, const CkptData& d)
{
    if (!path) return HP_ERR_INVALID_ARG;
    const size_t n = d.w.size();
    if (d.has_moments && (d.m.size() != n || d.v.size() != n)) return HP_ERR_INVALID_ARG;
    // written under a temporary name and renamed, so that a crash never
    // leaves a truncated file under the final name
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = fopen(tmp.c_str(), "wb");
    if (!f) return HP_ERR_IO;
    Header h;
    memcpy(h.magic, kMagic, 8);
    h.version = kVersion;
    h.arch = d.arch;
    h.n = (int64_t)n;
    h.step = d.step;
    h.moments = d.has_moments ? 1u : 0u;
    h.reserved = 0;
    Fnv fnv;
    bool ok = put(f, fnv, &h, sizeof(h)) && put(f, fnv, d.w.data(), n * 4);
    if (ok && d.has_moments) ok = put(f, fnv, d.m.data(), n * 4) && put(f, fnv, d.v.data(), n * 4);
    const uint64_t sum = fnv.h;
    ok = ok && fwrite(&sum, 1, 8, f) == 8;
    ok = (fclose(f) == 0) && ok;
    if (!ok || rename(tmp.c_str(), path) != 0) {
        remove(tmp.c_str());
        return HP_ERR_IO;
    }
    return HP_OK;
}

hp_status ckpt_read(const char* path, CkptData* d)
{
    if (!path || !d) return HP_ERR_INVALID_ARG;
    FILE* f = fopen(path, "rb");
    if (!f) return HP_ERR_IO;
    // the file's size first: a header is only trusted (and its arrays
    // allocated) when the file holds exactly what it announces
    int64_t size = -1;
    if (fseeko(f, 0, SEEK_END) == 0) size = (int64_t)ftello(f);
    if (size < 0 || fseeko(f, 0, SEEK_SET) != 0) {
        fclose(f);
        return HP_ERR_IO;
    }
    Header h;
    Fnv fnv;
    bool ok = get(f, fnv, &h, sizeof(h)) && memcmp(h.magic, kMagic, 8) == 0 &&
              h.version == kVersion && h.n > 0 && h.n < (int64_t)1 << 32 && h.moments <= 1 &&
              h.step >= 0 && h.step <= INT32_MAX &&
              size == (int64_t)sizeof(Header) + h.n * 4 * (h.moments ? 3 : 1) + 8;
    if (ok) {
        d->arch = h.arch;
        d->step = h.step;
        d->has_moments = h.moments == 1;
        d->w.assign((size_t)h.n, 0.0f);
        ok = get(f, fnv, d->w.data(), (size_t)h.n * 4);
        if (ok && d->has_moments) {
            d->m.assign((size_t)h.n, 0.0f);
            d->v.assign((size_t)h.n, 0.0f);
            ok = get(f, fnv, d->m.data(), (size_t)h.n * 4) &&
                 get(f, fnv, d->v.data(), (size_t)h.n * 4);
        }
    }
    uint64_t sum = 0;
    const uint64_t expect = fnv.h;
    ok = ok && fread(&sum, 1, 8, f) == 8 && sum == expect;
    // nothing may follow the checksum
    unsigned char extra;
    ok = ok && fread(&extra, 1, 1, f) == 0;
    fclose(f);
    return ok ? HP_OK : HP_ERR_IO;
}

}  // namespace hp
