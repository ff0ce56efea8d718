// Circuit text parser, gate table and lowering to controlled single-qubit
// updates.  The gate set follows Sec. 2-4: single-qubit gates, CNOT (Sec. 3)
// and CZ (Sec. 4), plus controlled phases and SWAP for the QFT.  The square
// roots SX, SY are the principal roots (eigenvalues 1 and i).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <sstream>

#include "sv_internal.h"

namespace sv {

namespace {
constexpr double kPi = 3.14159265358979323846;

Cplx c(double re, double im = 0.0) { return Cplx{re, im}; }
Cplx cis(double th) { return Cplx{std::cos(th), std::sin(th)}; }

bool is_two_qubit(const std::string &n) { return n == "CZ" || n == "CX" || n == "CP" || n == "SWAP"; }
}  // namespace

int gate_matrix(const std::string &name, const double *p, int np, Cplx *m) {
    const double h = 1.0 / std::sqrt(2.0);
    if (!is_two_qubit(name)) {
        for (int k = 0; k < 4; ++k) m[k] = c(0);
        if (name == "H") { m[0] = c(h); m[1] = c(h); m[2] = c(h); m[3] = c(-h); }
        else if (name == "X") { m[1] = c(1); m[2] = c(1); }
        else if (name == "Y") { m[1] = c(0, -1); m[2] = c(0, 1); }
        else if (name == "Z") { m[0] = c(1); m[3] = c(-1); }
        else if (name == "S") { m[0] = c(1); m[3] = c(0, 1); }
        else if (name == "SDG") { m[0] = c(1); m[3] = c(0, -1); }
        else if (name == "T") { m[0] = c(1); m[3] = cis(kPi / 4); }
        else if (name == "TDG") { m[0] = c(1); m[3] = cis(-kPi / 4); }
        else if (name == "SX") { m[0] = c(.5, .5); m[1] = c(.5, -.5); m[2] = c(.5, -.5); m[3] = c(.5, .5); }
        else if (name == "SXDG") { m[0] = c(.5, -.5); m[1] = c(.5, .5); m[2] = c(.5, .5); m[3] = c(.5, -.5); }
        else if (name == "SY") { m[0] = c(.5, .5); m[1] = c(-.5, -.5); m[2] = c(.5, .5); m[3] = c(.5, .5); }
        else if (name == "SYDG") { m[0] = c(.5, -.5); m[1] = c(.5, -.5); m[2] = c(-.5, .5); m[3] = c(.5, -.5); }
        else if (name == "P") { if (np != 1) return -1; m[0] = c(1); m[3] = cis(p[0]); }
        else if (name == "U") {
            if (np != 8) return -1;
            for (int k = 0; k < 4; ++k) m[k] = c(p[2 * k], p[2 * k + 1]);
        } else return -1;
        return 1;
    }
    for (int k = 0; k < 16; ++k) m[k] = c(0);
    // local index = bit(first qubit) + 2 * bit(second qubit)
    if (name == "CZ") { m[0] = c(1); m[5] = c(1); m[10] = c(1); m[15] = c(-1); }
    else if (name == "CP") { if (np != 1) return -1; m[0] = c(1); m[5] = c(1); m[10] = c(1); m[15] = cis(p[0]); }
    else if (name == "CX") { m[0] = c(1); m[10] = c(1); m[1 * 4 + 3] = c(1); m[3 * 4 + 1] = c(1); }
    else if (name == "SWAP") { m[0] = c(1); m[1 * 4 + 2] = c(1); m[2 * 4 + 1] = c(1); m[15] = c(1); }
    else return -1;
    return 2;
}

sv_status parse_circuit(const char *text, int n_expected, Circuit *out) {
    out->n = -1;
    out->instrs.clear();
    if (!text) {
        set_error("circuit text is NULL");
        return SV_ERR_ARG;
    }
    std::istringstream in(text);
    std::string line;
    int lineno = 0;
    while (std::getline(in, line)) {
        ++lineno;
        const size_t hash = line.find('#');
        if (hash != std::string::npos) line.resize(hash);
        std::istringstream ls(line);
        std::vector<std::string> tok;
        for (std::string t; ls >> t;) tok.push_back(t);
        if (tok.empty()) continue;
        if (tok[0] == "qubits") {
            if (tok.size() != 2) {
                set_error("line %d: bad 'qubits' line", lineno);
                return SV_ERR_PARSE;
            }
            out->n = std::atoi(tok[1].c_str());
            continue;
        }
        Instr ins;
        ins.name = tok[0];
        ins.nq = is_two_qubit(ins.name) ? 2 : 1;
        if (int(tok.size()) < 1 + ins.nq) {
            set_error("line %d: missing qubit", lineno);
            return SV_ERR_PARSE;
        }
        for (int k = 0; k < ins.nq; ++k) {
            char *end = nullptr;
            const long v = std::strtol(tok[1 + k].c_str(), &end, 10);
            if (!end || *end) {
                set_error("line %d: bad qubit '%s'", lineno, tok[1 + k].c_str());
                return SV_ERR_PARSE;
            }
            ins.q[k] = int(v);
        }
        ins.np = int(tok.size()) - 1 - ins.nq;
        if (ins.np > 8) {
            set_error("line %d: too many parameters", lineno);
            return SV_ERR_PARSE;
        }
        for (int k = 0; k < ins.np; ++k) {
            char *end = nullptr;
            ins.p[k] = std::strtod(tok[1 + ins.nq + k].c_str(), &end);
            if (!end || *end) {
                set_error("line %d: bad parameter '%s'", lineno, tok[1 + ins.nq + k].c_str());
                return SV_ERR_PARSE;
            }
        }
        Cplx m[16];
        if (gate_matrix(ins.name, ins.p, ins.np, m) < 0) {
            set_error("line %d: unknown gate or wrong parameter count '%s'", lineno, ins.name.c_str());
            return SV_ERR_PARSE;
        }
        out->instrs.push_back(ins);
    }
    if (out->n < 0) out->n = n_expected;
    if (n_expected >= 0 && out->n != n_expected) {
        set_error("circuit declares %d qubits, state has %d", out->n, n_expected);
        return SV_ERR_ARG;
    }
    for (size_t g = 0; g < out->instrs.size(); ++g) {
        const Instr &ins = out->instrs[g];
        for (int k = 0; k < ins.nq; ++k)
            if (ins.q[k] < 0 || ins.q[k] >= out->n) {
                set_error("gate %zu (%s): qubit %d out of range [0,%d)", g, ins.name.c_str(), ins.q[k], out->n);
                return SV_ERR_ARG;
            }
        if (ins.nq == 2 && ins.q[0] == ins.q[1]) {
            set_error("gate %zu (%s): repeated qubit", g, ins.name.c_str());
            return SV_ERR_ARG;
        }
    }
    return SV_OK;
}

std::vector<Gate1> lower_to_gate1(const Circuit &circ) {
    std::vector<Gate1> out;
    out.reserve(circ.instrs.size() + 8);
    Cplx m[16];
    for (const Instr &ins : circ.instrs) {
        Gate1 g{};
        if (ins.nq == 1) {
            gate_matrix(ins.name, ins.p, ins.np, m);
            g.target = ins.q[0];
            g.control = -1;
            for (int k = 0; k < 4; ++k) g.u[k] = m[k];
            out.push_back(g);
            continue;
        }
        const int a = ins.q[0], b = ins.q[1];
        if (ins.name == "SWAP") {
            gate_matrix("X", nullptr, 0, m);
            for (int k = 0; k < 4; ++k) g.u[k] = m[k];
            g.target = b; g.control = a; out.push_back(g);
            g.target = a; g.control = b; out.push_back(g);
            g.target = b; g.control = a; out.push_back(g);
            continue;
        }
        if (ins.name == "CZ") gate_matrix("Z", nullptr, 0, m);
        else if (ins.name == "CX") gate_matrix("X", nullptr, 0, m);
        else gate_matrix("P", ins.p, 1, m);  // CP
        for (int k = 0; k < 4; ++k) g.u[k] = m[k];
        g.target = b;
        g.control = a;
        out.push_back(g);
    }
    return out;
}

}  // namespace sv
