// Gate fusion for SV_MODE_FUSED: consecutive gates are grouped into blocks of
// at most k qubits (Sec. 2: a product of gates on k qubits is one 2^k x 2^k
// matrix), and each block's matrix is the ordered product of its gates,
// computed in FP64.  A gate joins the current block when all its qubits fit
// and no earlier gate that was left out shares a qubit with it (diagonal
// gates commute with each other and may pass one another).
#include <complex>

#include "plan.h"

namespace sv {

namespace {

using cd = std::complex<double>;

struct FInstr {
    uint64_t qmask;
    bool diag;
    int nq;
    int q[2];
    cd m[16];
};

// U <- G U on k local qubits (U: d x d row-major), G a 1- or 2-qubit gate on
// local qubits lq (matrix local index bit j <-> lq[j]).
void left_multiply(std::vector<cd> &U, int k, const FInstr &g, const int *lq) {
    const int d = 1 << k, gd = 1 << g.nq;
    uint32_t mask = 0;
    for (int j = 0; j < g.nq; ++j) mask |= 1u << lq[j];
    std::vector<cd> in(static_cast<size_t>(gd)), out(static_cast<size_t>(gd));
    for (int col = 0; col < d; ++col)
        for (int i = 0; i < d; ++i) {
            if (uint32_t(i) & mask) continue;
            for (int l = 0; l < gd; ++l) {
                int idx = i;
                for (int j = 0; j < g.nq; ++j)
                    if (l >> j & 1) idx |= 1 << lq[j];
                in[size_t(l)] = U[size_t(idx) * d + col];
            }
            for (int r = 0; r < gd; ++r) {
                cd acc = 0;
                for (int l = 0; l < gd; ++l) acc += g.m[r * gd + l] * in[size_t(l)];
                out[size_t(r)] = acc;
            }
            for (int l = 0; l < gd; ++l) {
                int idx = i;
                for (int j = 0; j < g.nq; ++j)
                    if (l >> j & 1) idx |= 1 << lq[j];
                U[size_t(idx) * d + col] = out[size_t(l)];
            }
        }
}

}  // namespace

std::vector<FusedBlock> fuse_blocks(const Circuit &c, int kmax) {
    std::vector<FInstr> F;
    F.reserve(c.instrs.size());
    for (const Instr &ins : c.instrs) {
        FInstr f{};
        f.nq = ins.nq;
        Cplx m[16];
        gate_matrix(ins.name, ins.p, ins.np, m);
        const int gd = 1 << ins.nq;
        f.diag = true;
        for (int r = 0; r < gd; ++r)
            for (int l = 0; l < gd; ++l) {
                f.m[r * gd + l] = cd(m[r * gd + l].re, m[r * gd + l].im);
                if (r != l && (m[r * gd + l].re != 0 || m[r * gd + l].im != 0)) f.diag = false;
            }
        f.qmask = 0;
        for (int j = 0; j < ins.nq; ++j) {
            f.q[j] = ins.q[j];
            f.qmask |= uint64_t(1) << ins.q[j];
        }
        F.push_back(f);
    }
    std::vector<int> pending(F.size());
    for (size_t i = 0; i < F.size(); ++i) pending[i] = int(i);
    std::vector<FusedBlock> blocks;
    while (!pending.empty()) {
        uint64_t Q = 0, bF = 0, bD = 0;
        std::vector<int> taken, rest;
        for (int idx : pending) {
            const FInstr &g = F[size_t(idx)];
            const bool conflict = g.diag ? (g.qmask & bF) != 0 : (g.qmask & (bF | bD)) != 0;
            if (conflict || __builtin_popcountll(Q | g.qmask) > kmax) {
                (g.diag ? bD : bF) |= g.qmask;
                rest.push_back(idx);
                continue;
            }
            Q |= g.qmask;
            taken.push_back(idx);
        }
        pending.swap(rest);
        FusedBlock b;
        int pos_of[64];
        for (int q = 0; q < 64; ++q)
            if (Q >> q & 1) {
                pos_of[q] = b.k;
                b.qubits[b.k++] = q;
            }
        const int d = 1 << b.k;
        std::vector<cd> U(size_t(d) * d, cd(0));
        for (int i = 0; i < d; ++i) U[size_t(i) * d + i] = 1;
        for (int idx : taken) {
            const FInstr &g = F[size_t(idx)];
            int lq[2];
            for (int j = 0; j < g.nq; ++j) lq[j] = pos_of[g.q[j]];
            left_multiply(U, b.k, g, lq);
        }
        b.U.resize(2 * U.size());
        for (size_t i = 0; i < U.size(); ++i) {
            b.U[2 * i] = U[i].real();
            b.U[2 * i + 1] = U[i].imag();
        }
        b.gates = int(taken.size());
        blocks.push_back(std::move(b));
    }
    return blocks;
}

}  // namespace sv
