// Host-side fermion -> qubit algebra (Sec. II-A, Eqs. (2)-(4); pool of
// Sec. III-E).
//
// Every mapping used here is a linear encoding of occupation bits over
// GF(2): qubit bits b = B n (mod 2), with B = I for Jordan-Wigner and the
// Fenwick-tree matrix for Bravyi-Kitaev (qubit k stores the parity of modes
// k+1-lowbit(k+1) .. k).  For any invertible B the creation operator is
//
//   a+_j = X^{c_j} Z^{p_j} (1 + Z^{q_j}) / 2
//        = 1/2 X^{c_j} Z^{p_j} + 1/2 X^{c_j} Z^{p_j ^ q_j},
//
// (Z factors act first) where c_j is column j of B (the qubits flipped when
// mode j fills), q_j is row j of B^-1 (so (-1)^{q_j . b} = (-1)^{n_j}) and
// p_j is the XOR of rows 0..j-1 of B^-1 (so (-1)^{p_j . b} is the fermionic
// sign of the modes below j).  Because p_j . c_j = 0 and q_j . c_j = 1, the
// annihilation operator is a_j = 1/2 X^c Z^p - 1/2 X^c Z^{p^q}.
//
// A term is held as (x, z, c) meaning c * X^x Z^z, which has real matrix
// elements: <r| X^x Z^z |col> = (-1)^{popcount(col & z)} when r = col ^ x.
// Products use X^a Z^b X^c Z^d = (-1)^{popcount(b & c)} X^{a^c} Z^{b^d}, so
// all coefficients stay real throughout.
#include "common.h"

#include <algorithm>
#include <cmath>
#include <mutex>

namespace tq {

namespace {

// Relabelled encodings: a base mapping (JW or BK) whose basis index is
// carried to another by an invertible linear map M over GF(2): bit i of the
// new index is the parity of the base index over rows[i] (a qubit
// permutation is the special case of one bit per row).  The encoding matrix
// becomes B' = M B.  Registered once per process, never removed; ids from
// TQ_MAPPING_FIRST_RELABELLED on.
struct Relabelled {
    int base;
    int N;
    std::vector<uint64_t> rows;
};
std::mutex g_relabel_mutex;
std::vector<Relabelled> g_relabelled;

bool find_relabelled(int mapping, Relabelled* out) {
    if (mapping < TQ_MAPPING_FIRST_RELABELLED) return false;
    std::lock_guard<std::mutex> lock(g_relabel_mutex);
    const size_t i = (size_t)(mapping - TQ_MAPPING_FIRST_RELABELLED);
    if (i >= g_relabelled.size()) return false;
    if (out) *out = g_relabelled[i];
    return true;
}

struct Enc {
    int N;
    std::vector<uint64_t> c;  // column j of B, as a qubit mask
    std::vector<uint64_t> q;  // row j of B^-1
    std::vector<uint64_t> p;  // xor of rows 0..j-1 of B^-1
};

int lowbit(int i) { return i & (-i); }

Enc make_encoding(int N, int mapping) {
    Enc e;
    e.N = N;
    Relabelled rl;
    const bool relabel = find_relabelled(mapping, &rl);
    if (relabel && rl.N != N)
        throw Error(TQ_EINVAL, "relabelled mapping registered for " + std::to_string(rl.N) + " qubits, used with " +
                                   std::to_string(N));
    const int base = relabel ? rl.base : mapping;
    // rows of B as masks over modes
    std::vector<uint64_t> base_rows(N, 0);
    for (int k = 0; k < N; ++k) {
        if (base == TQ_JW) {
            base_rows[k] = 1ull << k;
        } else {
            int lo = k + 1 - lowbit(k + 1);
            for (int i = lo; i <= k; ++i) base_rows[k] |= 1ull << i;
        }
    }
    // a relabelling combines the base rows: row i of B' = M B is the xor of
    // the base rows that row i of M selects
    std::vector<uint64_t> rows(N, 0);
    for (int i = 0; i < N; ++i) {
        if (!relabel) {
            rows[i] = base_rows[i];
            continue;
        }
        for (int k = 0; k < N; ++k)
            if ((rl.rows[i] >> k) & 1) rows[i] ^= base_rows[k];
    }
    e.c.assign(N, 0);
    for (int k = 0; k < N; ++k)
        for (int j = 0; j < N; ++j)
            if ((rows[k] >> j) & 1) e.c[j] |= 1ull << k;
    // invert B over GF(2) by Gauss-Jordan on [B | I]
    std::vector<uint64_t> a = rows, inv(N, 0);
    for (int k = 0; k < N; ++k) inv[k] = 1ull << k;
    for (int col = 0; col < N; ++col) {
        int piv = -1;
        for (int r = col; r < N; ++r)
            if ((a[r] >> col) & 1) { piv = r; break; }
        if (piv < 0) throw Error(TQ_ENUMERIC, "encoding matrix is singular");
        std::swap(a[piv], a[col]);
        std::swap(inv[piv], inv[col]);
        for (int r = 0; r < N; ++r)
            if (r != col && ((a[r] >> col) & 1)) { a[r] ^= a[col]; inv[r] ^= inv[col]; }
    }
    // inv[j] is row j of B^-1 as a mask over qubits
    e.q = inv;
    e.p.assign(N, 0);
    uint64_t acc = 0;
    for (int j = 0; j < N; ++j) { e.p[j] = acc; acc ^= inv[j]; }
    return e;
}

struct Term { uint64_t x, z; double c; };

inline int parity64(uint64_t v) { return __builtin_popcountll(v) & 1; }

// Ladder operator as two terms.
inline void ladder(const Enc& e, int j, bool create, Term out[2]) {
    out[0] = {e.c[j], e.p[j], 0.5};
    out[1] = {e.c[j], e.p[j] ^ e.q[j], create ? 0.5 : -0.5};
}

inline Term mul(const Term& a, const Term& b) {
    double s = parity64(a.z & b.x) ? -1.0 : 1.0;
    return {a.x ^ b.x, a.z ^ b.z, a.c * b.c * s};
}

// Expand coef * op_0 op_1 ... op_{m-1} (left to right) into `out`.
void expand(const Enc& e, double coef, const int* modes, const bool* create, int m,
            std::vector<Term>& out) {
    Term lad[4][2];
    for (int o = 0; o < m; ++o) ladder(e, modes[o], create[o], lad[o]);
    for (int choice = 0; choice < (1 << m); ++choice) {
        Term t = lad[0][choice & 1];
        for (int o = 1; o < m; ++o) t = mul(t, lad[o][(choice >> o) & 1]);
        t.c *= coef;
        out.push_back(t);
    }
}

// Sort by (x, z), merge like terms (summing in generation order), drop
// |c| <= rel * max|c|.
std::vector<PauliTerm> canonicalise(std::vector<Term>& t, double rel) {
    std::stable_sort(t.begin(), t.end(), [](const Term& a, const Term& b) {
        return a.x != b.x ? a.x < b.x : a.z < b.z;
    });
    std::vector<PauliTerm> merged;
    for (size_t i = 0; i < t.size();) {
        size_t j = i;
        double s = 0.0;
        while (j < t.size() && t[j].x == t[i].x && t[j].z == t[i].z) s += t[j++].c;
        merged.push_back({t[i].x, t[i].z, s});
        i = j;
    }
    double mx = 0.0;
    for (auto& m : merged) mx = std::max(mx, std::fabs(m.c));
    std::vector<PauliTerm> out;
    for (auto& m : merged)
        if (std::fabs(m.c) > rel * mx) out.push_back(m);
    return out;
}

}  // namespace

void check_mapping(int mapping) {
    if (mapping != TQ_JW && mapping != TQ_BK && !find_relabelled(mapping, nullptr))
        throw Error(TQ_EINVAL, "mapping must be TQ_JW, TQ_BK or an id from tq_mapping_relabelled / tq_mapping_linear");
}

namespace {
// Inverse over GF(2) of the N x N matrix with the given rows (bit j of
// rows[i] is entry (i, j)); false when singular.
bool gf2_inverse(std::vector<uint64_t> a, int N, std::vector<uint64_t>& inv) {
    inv.assign(N, 0);
    for (int k = 0; k < N; ++k) inv[k] = 1ull << k;
    for (int col = 0; col < N; ++col) {
        int piv = -1;
        for (int r = col; r < N; ++r)
            if ((a[r] >> col) & 1) { piv = r; break; }
        if (piv < 0) return false;
        std::swap(a[piv], a[col]);
        std::swap(inv[piv], inv[col]);
        for (int r = 0; r < N; ++r)
            if (r != col && ((a[r] >> col) & 1)) { a[r] ^= a[col]; inv[r] ^= inv[col]; }
    }
    return true;
}
}  // namespace

int register_linear(int base, int N, const uint64_t* rows) {
    if (base != TQ_JW && base != TQ_BK) throw Error(TQ_EINVAL, "base mapping must be TQ_JW or TQ_BK");
    if (N < 1 || N > 2 * TQ_MAX_SPATIAL) throw Error(TQ_EINVAL, "n_qubits out of range [1, 30]");
    if (!rows) throw Error(TQ_EINVAL, "null rows");
    const uint64_t full = (N == 64) ? ~0ull : ((1ull << N) - 1ull);
    for (int i = 0; i < N; ++i)
        if (rows[i] & ~full) throw Error(TQ_EINVAL, "a row selects a qubit beyond n_qubits");
    std::vector<uint64_t> r(rows, rows + N), inv;
    if (!gf2_inverse(r, N, inv)) throw Error(TQ_EINVAL, "the index map is not invertible over GF(2)");
    std::lock_guard<std::mutex> lock(g_relabel_mutex);
    for (size_t i = 0; i < g_relabelled.size(); ++i) {
        const Relabelled& x = g_relabelled[i];
        if (x.base == base && x.N == N && x.rows == r) return TQ_MAPPING_FIRST_RELABELLED + (int)i;
    }
    if (g_relabelled.size() >= 4096) throw Error(TQ_EINVAL, "too many relabelled mappings (4096)");
    g_relabelled.push_back({base, N, r});
    return TQ_MAPPING_FIRST_RELABELLED + (int)g_relabelled.size() - 1;
}

int register_relabelled(int base, int N, const int* order) {
    if (base != TQ_JW && base != TQ_BK) throw Error(TQ_EINVAL, "base mapping must be TQ_JW or TQ_BK");
    if (N < 1 || N > 2 * TQ_MAX_SPATIAL) throw Error(TQ_EINVAL, "n_qubits out of range [1, 30]");
    if (!order) throw Error(TQ_EINVAL, "null order");
    std::vector<int> seen(N, 0);
    for (int k = 0; k < N; ++k) {
        if (order[k] < 0 || order[k] >= N || seen[order[k]]) throw Error(TQ_EINVAL, "order is not a permutation of 0..n_qubits-1");
        seen[order[k]] = 1;
    }
    // qubit k at bit order[k]: row order[k] of M selects qubit k
    std::vector<uint64_t> rows(N, 0);
    for (int k = 0; k < N; ++k) rows[order[k]] = 1ull << k;
    return register_linear(base, N, rows.data());
}

namespace {
// rank over GF(2) of up to three masks
int gf2_rank(uint64_t a[3], int m) {
    int rank = 0;
    for (int bit = 0; bit < 64 && rank < m; ++bit) {
        int piv = -1;
        for (int i = rank; i < m; ++i)
            if ((a[i] >> bit) & 1) { piv = i; break; }
        if (piv < 0) continue;
        std::swap(a[piv], a[rank]);
        for (int i = 0; i < m; ++i)
            if (i != rank && ((a[i] >> bit) & 1)) a[i] ^= a[rank];
        ++rank;
    }
    return rank;
}
}  // namespace

std::vector<int> pool_sector_order(int n, int ne, int base, int low_bits) {
    if (base != TQ_JW && base != TQ_BK) throw Error(TQ_EINVAL, "base mapping must be TQ_JW or TQ_BK");
    const int N = 2 * n;
    if (low_bits < 0 || low_bits > N) throw Error(TQ_EINVAL, "low_bits out of range [0, 2 n_spatial]");
    const auto ex = excitations(n, ne);
    // every generator's support conditions (masks over the base qubits)
    struct Supp { int m; uint64_t e[3]; };
    std::vector<Supp> sup;
    for (const auto& x : ex) {
        const auto t = pauli_generator(x, N, base);
        const SignForm f = factor_generator(t);
        if (!f.ok) throw Error(TQ_ENUMERIC, "generator without a factored sign form");
        const SupportForm sf = support_form(f, t.front().x);
        Supp s{sf.m, {sf.e[0], sf.e[1], sf.e[2]}};
        sup.push_back(s);
    }
    // greedy: the next lowest index bit takes the qubit that keeps the most
    // support rows per touched segment of 2^(bits so far) amplitudes; a
    // support with conditions of rank r on those bits fills 2^-r of them
    std::vector<int> chosen;
    uint64_t mask = 0;
    for (int l = 0; l < low_bits; ++l) {
        int best = -1;
        double best_cost = 0.0;
        for (int q = 0; q < N; ++q) {
            if ((mask >> q) & 1) continue;
            const uint64_t mq = mask | (1ull << q);
            double cost = 0.0;
            for (const auto& s : sup) {
                uint64_t a[3] = {s.e[0] & mq, s.e[1] & mq, s.e[2] & mq};
                cost += std::ldexp(1.0, N - s.m + gf2_rank(a, s.m));
            }
            if (best < 0 || cost < best_cost) {
                best = q;
                best_cost = cost;
            }
        }
        chosen.push_back(best);
        mask |= 1ull << best;
    }
    std::vector<int> order(N, -1);
    int next = 0;
    for (int q : chosen) order[q] = next++;
    for (int q = 0; q < N; ++q)
        if (order[q] < 0) order[q] = next++;
    return order;
}

std::vector<uint64_t> pool_sector_basis(int n, int ne, int base, int low_bits) {
    if (base != TQ_JW && base != TQ_BK) throw Error(TQ_EINVAL, "base mapping must be TQ_JW or TQ_BK");
    const int N = 2 * n;
    if (n < 1 || n > TQ_MAX_SPATIAL) throw Error(TQ_EINVAL, "n_spatial out of range");
    if (low_bits < 0 || low_bits > N) throw Error(TQ_EINVAL, "low_bits out of range [0, 2 n_spatial]");
    const auto ex = excitations(n, ne);
    // every generator's support conditions (masks over the base index)
    struct Supp { int m; uint64_t e[3]; };
    std::vector<Supp> sup;
    for (const auto& x : ex) {
        const auto t = pauli_generator(x, N, base);
        const SignForm f = factor_generator(t);
        if (!f.ok) throw Error(TQ_ENUMERIC, "generator without a factored sign form");
        const SupportForm sf = support_form(f, t.front().x);
        sup.push_back(Supp{sf.m, {(uint64_t)sf.e[0], (uint64_t)sf.e[1], (uint64_t)sf.e[2]}});
    }
    const size_t G = sup.size();
    // candidates: every vector while 2^N x generators stays modest, else
    // the unit vectors and their pairwise sums
    std::vector<uint64_t> cand;
    if ((double)(1ull << N) * (double)std::max<size_t>(G, 1) <= (double)(1ull << 26)) {
        for (uint64_t v = 1; v < (1ull << N); ++v) cand.push_back(v);
    } else {
        for (int a = 0; a < N; ++a) {
            cand.push_back(1ull << a);
            for (int b = a + 1; b < N; ++b) cand.push_back((1ull << a) | (1ull << b));
        }
    }
    // greedy: new index bit l takes the vector v (independent of those before
    // it) that keeps the most support rows per touched segment of 2^(l+1)
    // amplitudes; a segment is a coset of V = span(chosen), and support S_k
    // fills |V cap K_k| of it, K_k the kernel of k's conditions.  In
    // syndrome terms: cost = sum_k |S_k| 2^rank_k, rank_k the rank of the
    // chosen vectors' syndromes (parities over k's condition masks).
    std::vector<uint8_t> span(G, 1);   // bit s: syndrome s lies in the span (starts with 0)
    std::vector<int> rank(G, 0);
    std::vector<uint64_t> basis;       // chosen vectors, in the order of the new index bits
    std::vector<uint64_t> echelon;     // reduced copies for the independence test
    auto reduce = [&](uint64_t v) {
        for (uint64_t r : echelon) {
            const uint64_t hb = 1ull << (63 - __builtin_clzll(r));
            if (v & hb) v ^= r;
        }
        return v;
    };
    auto add_echelon = [&](uint64_t v) {
        v = reduce(v);
        if (!v) return false;
        const uint64_t hb = 1ull << (63 - __builtin_clzll(v));
        for (auto& r : echelon)
            if (r & hb) r ^= v;
        echelon.push_back(v);
        std::sort(echelon.begin(), echelon.end(), [](uint64_t a, uint64_t b) { return a > b; });
        return true;
    };
    auto syndrome = [&](const Supp& s, uint64_t v) {
        int y = 0;
        for (int i = 0; i < s.m; ++i) y |= (__builtin_popcountll(v & s.e[i]) & 1) << i;
        return y;
    };
    for (int l = 0; l < low_bits; ++l) {
        uint64_t best = 0;
        double best_cost = 0.0;
        for (uint64_t v : cand) {
            if (!reduce(v)) continue;
            double cost = 0.0;
            for (size_t k = 0; k < G; ++k) {
                const int inside = (span[k] >> syndrome(sup[k], v)) & 1;
                cost += std::ldexp(1.0, N - sup[k].m + rank[k] + (inside ? 0 : 1));
            }
            if (best == 0 || cost < best_cost) {
                best = v;
                best_cost = cost;
            }
        }
        if (best == 0) break;   // no independent candidate left
        basis.push_back(best);
        add_echelon(best);
        for (size_t k = 0; k < G; ++k) {
            const int y = syndrome(sup[k], best);
            if (!((span[k] >> y) & 1)) {
                uint8_t grown = span[k];
                for (int s = 0; s < 8; ++s)
                    if ((span[k] >> s) & 1) grown |= (uint8_t)(1u << (s ^ y));
                span[k] = grown;
                ++rank[k];
            }
        }
    }
    // the remaining bits: unit vectors not yet spanned, in qubit order
    for (int q = 0; q < N && (int)basis.size() < N; ++q)
        if (add_echelon(1ull << q)) basis.push_back(1ull << q);
    // basis[i] is new index bit i in base coordinates: the columns of M^-1
    std::vector<uint64_t> crow(N, 0), m;
    for (int i = 0; i < N; ++i)
        for (int j = 0; j < N; ++j)
            if ((basis[i] >> j) & 1) crow[j] |= 1ull << i;
    if (!gf2_inverse(crow, N, m)) throw Error(TQ_ENUMERIC, "sector basis is singular");
    return m;   // rows of M: new bit i = parity(base index & m[i])
}

std::vector<PauliTerm> pauli_hamiltonian(int n, const double* h1, const double* g2,
                                         double e_const, int mapping) {
    if (n < 1 || n > TQ_MAX_SPATIAL) throw Error(TQ_EINVAL, "n_spatial out of range [1, 15]");
    if (!h1 || !g2) throw Error(TQ_EINVAL, "null integral array");
    check_mapping(mapping);
    const int N = 2 * n;
    Enc e = make_encoding(N, mapping);
    std::vector<Term> terms;
    terms.reserve(16ull * N * N * N * N / 4 + 4ull * N * N + 1);
    // one-body: h_PQ a+_P a_Q, equal spins
    for (int P = 0; P < N; ++P)
        for (int Q = 0; Q < N; ++Q) {
            if ((P & 1) != (Q & 1)) continue;
            double v = h1[(P >> 1) * n + (Q >> 1)];
            if (v == 0.0) continue;
            int modes[2] = {P, Q};
            bool cr[2] = {true, false};
            expand(e, v, modes, cr, 2, terms);
        }
    // two-body: 1/2 (PQ|RS) a+_P a+_R a_S a_Q, sigma_P = sigma_Q, sigma_R = sigma_S
    for (int P = 0; P < N; ++P)
        for (int Q = 0; Q < N; ++Q) {
            if ((P & 1) != (Q & 1)) continue;
            for (int R = 0; R < N; ++R)
                for (int S = 0; S < N; ++S) {
                    if ((R & 1) != (S & 1) || P == R || Q == S) continue;
                    size_t idx = (((size_t)(P >> 1) * n + (Q >> 1)) * n + (R >> 1)) * n + (S >> 1);
                    double v = g2[idx];
                    if (v == 0.0) continue;
                    int modes[4] = {P, R, S, Q};
                    bool cr[4] = {true, true, false, false};
                    expand(e, 0.5 * v, modes, cr, 4, terms);
                }
        }
    terms.push_back({0, 0, e_const});
    std::vector<PauliTerm> out = canonicalise(terms, 1e-12);
    for (auto& t : out)
        if (parity64(t.x & t.z))
            throw Error(TQ_ENUMERIC, "Hamiltonian term with an odd number of Y survived");
    return out;
}

std::vector<Excitation> excitations(int n, int ne) {
    if (n < 1 || n > TQ_MAX_SPATIAL) throw Error(TQ_EINVAL, "n_spatial out of range [1, 15]");
    const int N = 2 * n;
    if (ne < 0 || ne > N) throw Error(TQ_EINVAL, "n_electrons out of range [0, 2 n_spatial]");
    std::vector<Excitation> out;
    for (int i = 0; i < ne; ++i)
        for (int a = ne; a < N; ++a)
            if ((i & 1) == (a & 1)) out.push_back({{i, a, -1, -1}, 1});
    for (int i = 0; i < ne; ++i)
        for (int j = i + 1; j < ne; ++j)
            for (int a = ne; a < N; ++a)
                for (int b = a + 1; b < N; ++b)
                    if ((i & 1) + (j & 1) == (a & 1) + (b & 1)) out.push_back({{i, j, a, b}, 2});
    return out;
}

std::vector<PauliTerm> pauli_generator(const Excitation& ex, int N, int mapping) {
    check_mapping(mapping);
    Enc e = make_encoding(N, mapping);
    std::vector<Term> t;
    if (ex.order == 1) {
        int i = ex.idx[0], a = ex.idx[1];
        int m1[2] = {a, i}, m2[2] = {i, a};
        bool cr[2] = {true, false};
        expand(e, 1.0, m1, cr, 2, t);    // tau = a+_a a_i
        expand(e, -1.0, m2, cr, 2, t);   // -tau+ = -a+_i a_a
    } else {
        int i = ex.idx[0], j = ex.idx[1], a = ex.idx[2], b = ex.idx[3];
        int m1[4] = {a, b, j, i}, m2[4] = {i, j, b, a};
        bool cr[4] = {true, true, false, false};
        expand(e, 1.0, m1, cr, 4, t);    // tau = a+_a a+_b a_j a_i
        expand(e, -1.0, m2, cr, 4, t);   // -tau+ = -a+_i a+_j a_b a_a
    }
    return canonicalise(t, 1e-12);
}

uint64_t hf_index(int N, int ne, int mapping) {
    check_mapping(mapping);
    if (ne < 0 || ne > N) throw Error(TQ_EINVAL, "n_electrons out of range");
    Enc e = make_encoding(N, mapping);
    uint64_t b = 0;
    for (int P = 0; P < ne; ++P) b ^= e.c[P];
    return b;
}

std::vector<uint32_t> decode_rows(int N, int mapping) {
    check_mapping(mapping);
    Enc e = make_encoding(N, mapping);
    std::vector<uint32_t> r(N);
    for (int j = 0; j < N; ++j) r[j] = (uint32_t)e.q[j];
    return r;
}

uint64_t encode_occupation(int N, int mapping, uint64_t occ) {
    check_mapping(mapping);
    Enc e = make_encoding(N, mapping);
    uint64_t b = 0;
    for (int P = 0; P < N; ++P)
        if ((occ >> P) & 1) b ^= e.c[P];
    return b;
}

namespace {
long long choose(int n, int k) {
    if (k < 0 || k > n) return 0;
    long long r = 1;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

// The k-subset of colexicographic rank `rank`: the largest element c_k is
// the largest c with C(c, k) <= rank, and so on down.
std::vector<int> colex_unrank(long long rank, int k) {
    std::vector<int> out(k);
    for (int j = k; j >= 1; --j) {
        int c = j - 1;
        while (choose(c + 1, j) <= rank) ++c;
        out[j - 1] = c;
        rank -= choose(c, j);
    }
    return out;
}
}  // namespace

long long sector_dim(int n, int na, int nb) { return choose(n, na) * choose(n, nb); }

SectorSpec make_sector_spec(int n, int na, int nb, int mapping) {
    check_mapping(mapping);
    if (n < 1 || 2 * n > TQ_MAX_STATE_QUBITS) throw Error(TQ_EINVAL, "n_spatial out of range [1, 13]");
    if (na < 0 || na > n || nb < 0 || nb > n) throw Error(TQ_EINVAL, "n_alpha, n_beta out of range [0, n_spatial]");
    SectorSpec s{};
    s.n = n;
    s.na = na;
    s.nb = nb;
    s.nq = 2 * n;
    s.mapping = mapping;
    auto rows = decode_rows(2 * n, mapping);
    for (int j = 0; j < 2 * n; ++j) s.dec[j] = rows[j];
    for (int i = 0; i < 16; ++i)
        for (int j = 0; j < 16; ++j) s.binom[i][j] = (int)choose(i, j);
    return s;
}

std::vector<uint32_t> sector_basis(const SectorSpec& s) {
    const long long da = choose(s.n, s.na), db = choose(s.n, s.nb);
    const Enc e = make_encoding(s.nq, s.mapping);
    // qubit-space images of the alpha and beta halves (the encoding is linear)
    std::vector<uint64_t> qa((size_t)da), qb((size_t)db);
    for (long long r = 0; r < da; ++r)
        for (int p : colex_unrank(r, s.na)) qa[(size_t)r] ^= e.c[2 * p];
    for (long long r = 0; r < db; ++r)
        for (int p : colex_unrank(r, s.nb)) qb[(size_t)r] ^= e.c[2 * p + 1];
    std::vector<uint32_t> out((size_t)(da * db));
    for (long long ra = 0; ra < da; ++ra)
        for (long long rb = 0; rb < db; ++rb) out[(size_t)(ra * db + rb)] = (uint32_t)(qa[(size_t)ra] ^ qb[(size_t)rb]);
    return out;
}

// ---------------------------------------------------------------------------
// Commuting families of the pool (Sec. III-F, Algorithm 1).

bool generators_commute(const PauliTerm* a, int na, const PauliTerm* b, int nb, int mode) {
    if (mode == TQ_COMMUTE_QWC) {
        // every pair of strings equal or identity on each qubit they share
        for (int i = 0; i < na; ++i)
            for (int j = 0; j < nb; ++j) {
                const uint64_t both = (a[i].x | a[i].z) & (b[j].x | b[j].z);
                if (((a[i].x ^ b[j].x) | (a[i].z ^ b[j].z)) & both) return false;
            }
        return true;
    }
    // [A, B] = sum over anticommuting string pairs of
    //   2 c_a c_b X^xa Z^za X^xb Z^zb = 2 c_a c_b (-1)^{za.xb} X^(xa^xb) Z^(za^zb),
    // summed per product string; the coefficients are dyadic, so the sums are exact
    std::vector<PauliTerm> acc;
    for (int i = 0; i < na; ++i)
        for (int j = 0; j < nb; ++j) {
            const int s1 = parity64(a[i].z & b[j].x), s2 = parity64(b[j].z & a[i].x);
            if (s1 == s2) continue;
            const uint64_t x = a[i].x ^ b[j].x, z = a[i].z ^ b[j].z;
            const double v = 2.0 * a[i].c * b[j].c * (s1 ? -1.0 : 1.0);
            bool found = false;
            for (auto& t : acc)
                if (t.x == x && t.z == z) {
                    t.c += v;
                    found = true;
                    break;
                }
            if (!found) acc.push_back({x, z, v});
        }
    for (const auto& t : acc)
        if (std::fabs(t.c) > 1e-12) return false;
    return true;
}

std::vector<int> greedy_families(int M, const std::vector<std::vector<int>>& nbr) {
    std::vector<int> order(M);
    for (int v = 0; v < M; ++v) order[v] = v;
    // largest degree first; equal degrees keep pool order
    std::stable_sort(order.begin(), order.end(),
                     [&](int u, int v) { return nbr[u].size() > nbr[v].size(); });
    std::vector<int> family(M, -1);
    int K = 0;
    std::vector<int> taken;
    for (int v : order) {
        taken.assign(K + 1, 0);
        for (int u : nbr[v])
            if (family[u] >= 0) taken[family[u]] = 1;
        int f = 0;
        while (taken[f]) ++f;           // lowest family with no neighbour (K: a new one)
        family[v] = f;
        if (f == K) ++K;
    }
    return family;
}

std::vector<int> pool_families(const std::vector<PauliTerm>& terms, const std::vector<int>& nterm, int mode) {
    if (mode != TQ_COMMUTE_FULL && mode != TQ_COMMUTE_QWC) throw Error(TQ_EINVAL, "mode must be TQ_COMMUTE_FULL or TQ_COMMUTE_QWC");
    const int M = (int)nterm.size();
    std::vector<std::vector<int>> nbr(M);
    for (int i = 0; i < M; ++i)
        for (int j = i + 1; j < M; ++j)
            if (!generators_commute(&terms[8 * i], nterm[i], &terms[8 * j], nterm[j], mode)) {
                nbr[i].push_back(j);
                nbr[j].push_back(i);
            }
    return greedy_families(M, nbr);
}

// Factor a generator's sign function (see common.h, SignForm).  The z masks
// of its 2^m terms form an affine space z0 ^ span(d_1..d_m); when the
// coefficients are c0 / 2^m * prod_i (-1)^{a_i t_i} (a = coordinates in that
// basis) the sum collapses to c0 (-1)^{col.z0} prod_i [col.d_i == t_i].
SignForm factor_generator(const std::vector<PauliTerm>& t) {
    SignForm f{};
    const int K = (int)t.size();
    int m = 0;
    while ((1 << m) < K) ++m;
    if ((1 << m) != K || m > 3) return f;  // not factorable -> generic path
    for (auto& x : t)
        if (x.x != t[0].x) return f;
    // basis of {z_p ^ z0} by elimination, remembering pivot bits
    const uint64_t z0 = t[0].z;
    std::vector<uint64_t> basis;
    std::vector<int> pivot;
    for (int p = 1; p < K && (int)basis.size() < m; ++p) {
        uint64_t v = t[p].z ^ z0;
        for (size_t i = 0; i < basis.size(); ++i)
            if ((v >> pivot[i]) & 1) v ^= basis[i];
        if (v) {
            int pb = 63 - __builtin_clzll(v);
            for (size_t i = 0; i < basis.size(); ++i)
                if ((basis[i] >> pb) & 1) basis[i] ^= v;
            basis.push_back(v);
            pivot.push_back(pb);
        }
    }
    if ((int)basis.size() != m) return f;
    const double c0 = t[0].c * (double)K;
    // coordinates of each term, and the implied signs t_i from unit vectors
    auto coords = [&](uint64_t z) {
        uint64_t v = z ^ z0;
        int a = 0;
        for (size_t i = 0; i < basis.size(); ++i)
            if ((v >> pivot[i]) & 1) { v ^= basis[i]; a |= 1 << i; }
        return v ? -1 : a;
    };
    int tbits = 0;
    std::vector<int> coord(K);
    for (int p = 0; p < K; ++p) {
        coord[p] = coords(t[p].z);
        if (coord[p] < 0) return f;
    }
    for (int p = 0; p < K; ++p)
        for (int i = 0; i < m; ++i)
            if (coord[p] == (1 << i) && t[p].c * c0 < 0) tbits |= 1 << i;
    for (int p = 0; p < K; ++p) {
        int par = __builtin_popcount(coord[p] & tbits) & 1;
        double expect = c0 / (double)K * (par ? -1.0 : 1.0);
        if (t[p].c != expect) return f;
    }
    f.ok = 1;
    f.m = m;
    f.c0 = c0;
    f.z0 = z0;
    for (int i = 0; i < m; ++i) f.d[i] = basis[i];
    f.t = tbits;
    return f;
}

SupportForm support_form(const SignForm& f, uint64_t x) {
    // conditions on col = r ^ x become conditions on r with flipped targets
    SupportForm s{};
    s.m = f.m;
    uint64_t e[3] = {f.d[0], f.d[1], f.d[2]};
    int t[3];
    for (int i = 0; i < f.m; ++i)
        t[i] = ((f.t >> i) & 1) ^ (__builtin_popcountll(x & e[i]) & 1);
    // reduce: pivot = highest set bit, eliminated from every other row
    int piv[3] = {0, 0, 0};
    for (int i = 0; i < f.m; ++i) {
        int best = i;
        for (int j = i + 1; j < f.m; ++j)
            if (e[j] > e[best]) best = j;
        std::swap(e[i], e[best]);
        std::swap(t[i], t[best]);
        if (e[i] == 0) throw Error(TQ_ENUMERIC, "degenerate generator support");
        piv[i] = 63 - __builtin_clzll(e[i]);
        for (int j = 0; j < f.m; ++j)
            if (j != i && ((e[j] >> piv[i]) & 1)) {
                e[j] ^= e[i];
                t[j] ^= t[i];
            }
    }
    // order by ascending pivot
    int ord[3] = {0, 1, 2};
    std::sort(ord, ord + f.m, [&](int a, int b) { return piv[a] < piv[b]; });
    for (int i = 0; i < f.m; ++i) {
        s.p[i] = piv[ord[i]];
        s.e[i] = e[ord[i]];
        s.target |= t[ord[i]] << i;
    }
    // pair representative bit: if every set bit of x were a pivot, the
    // conditions parity(x & e[i]) == 0 (x maps the support to itself) would
    // force x = 0
    s.h = -1;
    for (int bit = 63; bit >= 0 && s.h < 0; --bit) {
        bool pivot = false;
        for (int i = 0; i < f.m; ++i) pivot = pivot || s.p[i] == bit;
        if (((x >> bit) & 1) && !pivot) s.h = bit;
    }
    if (s.h < 0) throw Error(TQ_ENUMERIC, "generator X-mask has no free bit");
    s.hp = s.h;
    for (int i = 0; i < f.m; ++i) s.hp -= s.p[i] < s.h;
    return s;
}

}  // namespace tq
