// Host I/O: FCIDUMP integral files and state checkpoints.
//
// The paper's molecular integrals are not available; real ones come in the
// common FCIDUMP text form: a Fortran namelist header (&FCI NORB=n,
// NELEC=ne, MS2=m, ... terminated by &END or /), then one integral per line,
// "value i j k l" with 1-based orbitals: all four non-zero -> the chemist
// integral (ij|kl); k = l = 0 -> h_ij; all zero -> the core energy; other
// patterns (orbital energies) are skipped.  Real orbitals give (ij|kl) the
// 8-fold symmetry and h the 2-fold one, so a file may list one member of
// each class; the reader fills every member.  Values may carry a Fortran D
// exponent.
//
// A state checkpoint is a 40-byte header (magic "TQSTATE1", then int32
// precision, qubits, sector flag, n_alpha, n_beta, 0, and int64 amplitude
// count) followed by the amplitudes as stored on the device.
#include "host_util.h"

#include <cctype>
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <sstream>
#include <string>
#include <vector>

using namespace tq;

namespace {

std::string upper(std::string s) {
    for (auto& ch : s) ch = (char)std::toupper((unsigned char)ch);
    return s;
}

// integer after "KEY=" in the header, or `fallback` when absent
int header_int(const std::string& up, const char* key, int fallback, bool required) {
    size_t pos = 0;
    const std::string k(key);
    while ((pos = up.find(k, pos)) != std::string::npos) {
        const bool word_start = pos == 0 || !std::isalnum((unsigned char)up[pos - 1]);
        size_t q = pos + k.size();
        while (q < up.size() && std::isspace((unsigned char)up[q])) ++q;
        if (word_start && q < up.size() && up[q] == '=') {
            ++q;
            while (q < up.size() && std::isspace((unsigned char)up[q])) ++q;
            char* end = nullptr;
            const long v = std::strtol(up.c_str() + q, &end, 10);
            if (end == up.c_str() + q) throw Error(TQ_EINVAL, std::string("FCIDUMP: no value for ") + key);
            return (int)v;
        }
        pos += k.size();
    }
    if (required) throw Error(TQ_EINVAL, std::string("FCIDUMP: header has no ") + key);
    return fallback;
}

struct Fcidump {
    int n = 0, ne = 0, ms2 = 0;
    std::string body;
};

Fcidump parse_header(const char* path) {
    std::ifstream f(path);
    if (!f) throw Error(TQ_EINVAL, std::string("cannot open ") + path);
    std::stringstream ss;
    ss << f.rdbuf();
    const std::string text = ss.str();
    const std::string up = upper(text);
    const size_t start = up.find("&FCI");
    if (start == std::string::npos) throw Error(TQ_EINVAL, "FCIDUMP: no &FCI header");
    size_t stop = up.find("&END", start);
    size_t after = stop == std::string::npos ? std::string::npos : stop + 4;
    const size_t slash = up.find('/', start);
    if (slash != std::string::npos && (stop == std::string::npos || slash < stop)) after = slash + 1;
    if (after == std::string::npos) throw Error(TQ_EINVAL, "FCIDUMP: header is not terminated");
    const std::string head = up.substr(start, after - start);
    Fcidump d;
    d.n = header_int(head, "NORB", 0, true);
    d.ne = header_int(head, "NELEC", 0, true);
    d.ms2 = header_int(head, "MS2", 0, false);
    if (d.n < 1 || d.n > TQ_MAX_SPATIAL) throw Error(TQ_EINVAL, "FCIDUMP: NORB out of range [1, 15]");
    if (d.ne < 0 || d.ne > 2 * d.n) throw Error(TQ_EINVAL, "FCIDUMP: NELEC out of range");
    d.body = text.substr(after);
    for (auto& ch : d.body)
        if (ch == 'D' || ch == 'd') ch = 'E';
    return d;
}

}  // namespace

extern "C" int tq_read_fcidump(const char* path, int* n_spatial, int* n_electrons, int* ms2, double* e_core,
                               double* h1, double* g2, int capacity_n) {
    API_BEGIN
    TQ_REQUIRE(path != nullptr, "null path");
    Fcidump d = parse_header(path);
    if (n_spatial) *n_spatial = d.n;
    if (n_electrons) *n_electrons = d.ne;
    if (ms2) *ms2 = d.ms2;
    if (!h1 && !g2 && !e_core) return TQ_OK;          // header only
    TQ_REQUIRE(!(h1 || g2) || capacity_n >= d.n, "capacity_n is smaller than NORB");
    const int n = d.n;
    const size_t n2 = (size_t)n * n;
    if (h1) std::memset(h1, 0, n2 * sizeof(double));
    if (g2) std::memset(g2, 0, n2 * n2 * sizeof(double));
    double core = 0.0;
    std::istringstream in(d.body);
    double v;
    long i, j, k, l;
    while (in >> v >> i >> j >> k >> l) {
        TQ_REQUIRE(i >= 0 && j >= 0 && k >= 0 && l >= 0 && i <= n && j <= n && k <= n && l <= n,
                   "FCIDUMP: orbital index out of range");
        if (i && j && k && l) {
            if (!g2) continue;
            const long o[8][4] = {{i, j, k, l}, {j, i, k, l}, {i, j, l, k}, {j, i, l, k},
                                  {k, l, i, j}, {l, k, i, j}, {k, l, j, i}, {l, k, j, i}};
            for (const auto& q : o)
                g2[(((size_t)(q[0] - 1) * n + (q[1] - 1)) * n + (q[2] - 1)) * n + (q[3] - 1)] = v;
        } else if (i && j && !k && !l) {
            if (!h1) continue;
            h1[(size_t)(i - 1) * n + (j - 1)] = v;
            h1[(size_t)(j - 1) * n + (i - 1)] = v;
        } else if (!i && !j && !k && !l) {
            core = v;
        }
    }
    TQ_REQUIRE(in.eof(), "FCIDUMP: malformed integral line");
    if (e_core) *e_core = core;
    API_END
}

extern "C" int tq_write_fcidump(const char* path, int n_spatial, int n_electrons, int ms2, const double* h1,
                                const double* g2, double e_core, double tol) {
    API_BEGIN
    TQ_REQUIRE(path && h1 && g2, "null argument");
    TQ_REQUIRE(n_spatial >= 1 && n_spatial <= TQ_MAX_SPATIAL, "n_spatial out of range [1, 15]");
    TQ_REQUIRE(std::isfinite(tol) && tol >= 0.0, "tol must be finite and >= 0");
    const int n = n_spatial;
    FILE* f = std::fopen(path, "w");
    TQ_REQUIRE(f != nullptr, std::string("cannot open ") + path);
    std::fprintf(f, " &FCI NORB=%d,NELEC=%d,MS2=%d,\n  ORBSYM=", n, n_electrons, ms2);
    for (int i = 0; i < n; ++i) std::fprintf(f, "1,");
    std::fprintf(f, "\n  ISYM=1,\n &END\n");
    // one member of each symmetry class: i >= j, k >= l, pair(ij) >= pair(kl)
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j)
            for (int k = 0; k < n; ++k)
                for (int l = 0; l <= k; ++l) {
                    if (i * (i + 1) / 2 + j < k * (k + 1) / 2 + l) continue;
                    const double v = g2[(((size_t)i * n + j) * n + k) * n + l];
                    if (std::fabs(v) > tol) std::fprintf(f, "%24.16E %4d %4d %4d %4d\n", v, i + 1, j + 1, k + 1, l + 1);
                }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j <= i; ++j) {
            const double v = h1[(size_t)i * n + j];
            if (std::fabs(v) > tol) std::fprintf(f, "%24.16E %4d %4d    0    0\n", v, i + 1, j + 1);
        }
    std::fprintf(f, "%24.16E    0    0    0    0\n", e_core);
    const bool ok = std::fclose(f) == 0;
    TQ_REQUIRE(ok, "write failed");
    API_END
}

namespace {

struct StateHeader {
    char magic[8];
    int32_t prec, nq, sector, na, nb, pad;
    int64_t D;
};
static_assert(sizeof(StateHeader) == 40, "state header layout");

}  // namespace

extern "C" int tq_state_save(const tq_state* s, const char* path) {
    API_BEGIN
    TQ_REQUIRE(s && path, "null argument");
    TQ_CUDA(cudaSetDevice(s->device));
    const size_t bytes = (size_t)s->D * (s->prec == TQ_C128 ? 16 : 8);
    std::vector<unsigned char> buf(bytes);
    TQ_CUDA(cudaDeviceSynchronize());
    TQ_CUDA(cudaMemcpy(buf.data(), s->data, bytes, cudaMemcpyDeviceToHost));
    StateHeader h{};
    std::memcpy(h.magic, "TQSTATE1", 8);
    h.prec = s->prec;
    h.nq = s->nq;
    h.sector = s->sector;
    h.na = s->n_alpha;
    h.nb = s->n_beta;
    h.D = s->D;
    FILE* f = std::fopen(path, "wb");
    TQ_REQUIRE(f != nullptr, std::string("cannot open ") + path);
    const bool ok = std::fwrite(&h, sizeof(h), 1, f) == 1 && std::fwrite(buf.data(), 1, bytes, f) == bytes;
    const bool closed = std::fclose(f) == 0;
    TQ_REQUIRE(ok && closed, "write failed");
    API_END
}

extern "C" int tq_state_load(tq_state* s, const char* path) {
    API_BEGIN
    TQ_REQUIRE(s && path, "null argument");
    FILE* f = std::fopen(path, "rb");
    TQ_REQUIRE(f != nullptr, std::string("cannot open ") + path);
    StateHeader h{};
    const bool got = std::fread(&h, sizeof(h), 1, f) == 1;
    const bool match = got && std::memcmp(h.magic, "TQSTATE1", 8) == 0 && h.prec == s->prec && h.nq == s->nq &&
                       h.sector == s->sector && h.na == s->n_alpha && h.nb == s->n_beta && h.D == s->D;
    if (!match) std::fclose(f);
    TQ_REQUIRE(got && std::memcmp(h.magic, "TQSTATE1", 8) == 0, "not a state checkpoint");
    TQ_REQUIRE(match, "checkpoint does not match the state (precision, qubits or sector)");
    const size_t bytes = (size_t)s->D * (s->prec == TQ_C128 ? 16 : 8);
    std::vector<unsigned char> buf(bytes);
    const bool ok = std::fread(buf.data(), 1, bytes, f) == bytes;
    std::fclose(f);
    TQ_REQUIRE(ok, "checkpoint is truncated");
    TQ_CUDA(cudaSetDevice(s->device));
    TQ_CUDA(cudaDeviceSynchronize());
    TQ_CUDA(cudaMemcpy(s->data, buf.data(), bytes, cudaMemcpyHostToDevice));
    API_END
}
