// Factor files: a versioned, checksummed container for the factors of one
// 1D butterfly factorization in the canonical layout of bf_plan_create, so a
// factorization built once (the construction of Sec. 3 costs far more than an
// apply) can be stored and planned again later.  Host code only.
//
// Layout (little-endian):
//   0  char[8] magic "BFLYFAC" + '\0'
//   8  u32     version (1)
//  12  u32     dtype (BF_C64 or BF_C128)
//  16  i32     L, leaf, r
//  28  u32     0
//  32  u64     payload bytes
//  40  u32     CRC-32 of the payload
//  44  u32     CRC-32 of bytes 0..43
//  48  16 zero bytes
//  64  payload: VL, H[0..h-1], S, G[0..h-1], UL, each in canonical order and
//      the file's dtype (S real: float for BF_C64, double for BF_C128; S
//      followed by zero bytes up to a multiple of 8, so every array after it
//      stays 8-byte aligned).
// The checksum is the CRC-32 of ISO-HDLC / IEEE 802.3 (reflected polynomial
// 0xEDB88320, initial value and final xor 0xFFFFFFFF; check value 0xCBF43926
// for the nine bytes "123456789"), computed eight bytes per step with eight
// lookup tables derived from the polynomial.

#include "bfly.h"

#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <vector>

namespace {

constexpr uint32_t kVersion = 1;
constexpr size_t kHeaderBytes = 64;
const char kMagic[8] = {'B', 'F', 'L', 'Y', 'F', 'A', 'C', '\0'};

struct CrcTables {
    uint32_t t[8][256];
    CrcTables() {
        for (uint32_t i = 0; i < 256; ++i) {
            uint32_t c = i;
            for (int k = 0; k < 8; ++k) c = (c & 1u) ? (c >> 1) ^ 0xEDB88320u : c >> 1;
            t[0][i] = c;
        }
        for (uint32_t i = 0; i < 256; ++i)
            for (int k = 1; k < 8; ++k) t[k][i] = (t[k - 1][i] >> 8) ^ t[0][t[k - 1][i] & 0xFFu];
    }
};
const CrcTables &crc_tables() {
    static const CrcTables tables;
    return tables;
}

// Running CRC-32 (pass the previous return value; start from 0).
uint32_t crc32_update(uint32_t crc, const unsigned char *p, size_t n) {
    const CrcTables &T = crc_tables();
    uint32_t c = ~crc;
    while (n >= 8) {
        const uint32_t lo = (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
        const uint32_t hi = (uint32_t)p[4] | ((uint32_t)p[5] << 8) | ((uint32_t)p[6] << 16) | ((uint32_t)p[7] << 24);
        c ^= lo;
        c = T.t[7][c & 0xFFu] ^ T.t[6][(c >> 8) & 0xFFu] ^ T.t[5][(c >> 16) & 0xFFu] ^ T.t[4][c >> 24] ^
            T.t[3][hi & 0xFFu] ^ T.t[2][(hi >> 8) & 0xFFu] ^ T.t[1][(hi >> 16) & 0xFFu] ^ T.t[0][hi >> 24];
        p += 8;
        n -= 8;
    }
    while (n--) c = T.t[0][(c ^ *p++) & 0xFFu] ^ (c >> 8);
    return ~c;
}

uint32_t rd32(const unsigned char *p) {
    return (uint32_t)p[0] | ((uint32_t)p[1] << 8) | ((uint32_t)p[2] << 16) | ((uint32_t)p[3] << 24);
}
uint64_t rd64(const unsigned char *p) { return (uint64_t)rd32(p) | ((uint64_t)rd32(p + 4) << 32); }

struct FileInfo {
    int dtype = 0, L = 0, leaf = 0, r = 0;
    uint64_t payload = 0;
    uint32_t crc = 0;
};

// Bytes of S in the payload (padded to a multiple of 8).
uint64_t s_bytes(const FileInfo &f) {
    const uint64_t m = 1ull << (f.L / 2);
    return (m * m * f.r * (f.dtype == BF_C64 ? 4 : 8) + 7) & ~7ull;
}

// Payload bytes the shape implies, or 0 if the shape is not one a plan could hold.
uint64_t payload_bytes(const FileInfo &f) {
    if (f.L < 0 || f.L > 24 || (f.L & 1) || f.leaf < 1 || f.leaf > 64 || f.r < 1 || f.r > 32) return 0;
    const uint64_t ce = f.dtype == BF_C64 ? 8 : 16;
    const uint64_t nb = 1ull << f.L, h = (uint64_t)f.L / 2;
    return 2 * nb * f.leaf * f.r * ce + 2 * h * nb * f.r * 2 * f.r * ce + s_bytes(f);
}

// Reads and checks the header; BF_OK, BF_ERR_CORRUPT or BF_ERR_UNSUPPORTED.
bf_status read_header(FILE *fp, FileInfo &f) {
    unsigned char h[kHeaderBytes];
    if (std::fread(h, 1, kHeaderBytes, fp) != kHeaderBytes) return BF_ERR_CORRUPT;
    if (std::memcmp(h, kMagic, 8) != 0) return BF_ERR_CORRUPT;
    if (crc32_update(0, h, 44) != rd32(h + 44)) return BF_ERR_CORRUPT;
    if (rd32(h + 8) != kVersion) return BF_ERR_UNSUPPORTED;
    f.dtype = (int)rd32(h + 12);
    f.L = (int)rd32(h + 16);
    f.leaf = (int)rd32(h + 20);
    f.r = (int)rd32(h + 24);
    f.payload = rd64(h + 32);
    f.crc = rd32(h + 40);
    if (f.dtype != BF_C64 && f.dtype != BF_C128) return BF_ERR_CORRUPT;
    const uint64_t need = payload_bytes(f);
    if (need == 0 || f.payload != need) return BF_ERR_CORRUPT;
    return BF_OK;
}

// Reads the payload into `buf` (if not null) in chunks, checking its CRC and
// that the file ends exactly after it.
bf_status read_payload(FILE *fp, const FileInfo &f, unsigned char *buf) {
    std::vector<unsigned char> scratch;
    const size_t chunk = 64u << 20;
    if (!buf) scratch.resize(chunk);
    uint32_t crc = 0;
    uint64_t done = 0;
    while (done < f.payload) {
        const size_t n = (size_t)std::min<uint64_t>(chunk, f.payload - done);
        unsigned char *dst = buf ? buf + done : scratch.data();
        if (std::fread(dst, 1, n, fp) != n) return BF_ERR_CORRUPT;   // truncated
        crc = crc32_update(crc, dst, n);
        done += n;
    }
    if (std::fgetc(fp) != EOF) return BF_ERR_CORRUPT;                // trailing bytes
    return crc == f.crc ? BF_OK : BF_ERR_CORRUPT;
}

}  // namespace

extern "C" {

unsigned int bf_crc32(const void *data, size_t bytes, unsigned int crc) {
    return data || bytes == 0 ? crc32_update(crc, static_cast<const unsigned char *>(data), bytes) : crc;
}

bf_status bf_factor_file_check(const char *path, bf_desc *desc, int *dtype) {
    if (!path) return BF_ERR_INVALID;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return BF_ERR_INVALID;
    FileInfo f;
    bf_status st = read_header(fp, f);
    if (st == BF_OK) st = read_payload(fp, f, nullptr);
    std::fclose(fp);
    if (st == BF_OK) {
        if (desc) {
            desc->L = f.L;
            desc->leaf = f.leaf;
            desc->r = f.r;
            desc->nrhs_max = 0;
        }
        if (dtype) *dtype = f.dtype;
    }
    return st;
}

bf_status bf_plan_create_from_file(bf_plan *plan, const char *path, int nrhs_max, cudaStream_t stream) {
    if (!plan) return BF_ERR_INVALID;
    *plan = nullptr;
    if (!path || nrhs_max < 1) return BF_ERR_INVALID;
    FILE *fp = std::fopen(path, "rb");
    if (!fp) return BF_ERR_INVALID;
    FileInfo f;
    bf_status st = read_header(fp, f);
    unsigned char *buf = nullptr;
    if (st == BF_OK) {
        buf = static_cast<unsigned char *>(std::malloc((size_t)f.payload));
        st = buf ? read_payload(fp, f, buf) : BF_ERR_NOMEM;
    }
    std::fclose(fp);
    if (st != BF_OK) {
        std::free(buf);
        return st;
    }
    const size_t ce = f.dtype == BF_C64 ? 8 : 16;
    const size_t nb = (size_t)1 << f.L, h = (size_t)f.L / 2;
    const size_t leaf_bytes = nb * f.leaf * f.r * ce, level_bytes = nb * f.r * 2 * f.r * ce;
    std::vector<const void *> H(h ? h : 1, nullptr), G(h ? h : 1, nullptr);
    size_t off = 0;
    const void *VL = buf + off;
    off += leaf_bytes;
    for (size_t t = 0; t < h; ++t, off += level_bytes) H[t] = buf + off;
    const void *S = buf + off;
    off += (size_t)s_bytes(f);
    for (size_t t = 0; t < h; ++t, off += level_bytes) G[t] = buf + off;
    const void *UL = buf + off;
    bf_desc d{f.L, f.leaf, f.r, nrhs_max};
    bf_factors fac;
    fac.dtype = f.dtype;
    fac.VL = VL;
    fac.H = H.data();
    fac.S = S;
    fac.G = G.data();
    fac.UL = UL;
    st = bf_plan_create(plan, &d, &fac, stream);
    std::free(buf);
    return st;
}

}  // extern "C"
