/*
 * oracle.c -- plain, slow CPU reference for the state-vector simulator.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * helper with the CUDA library; it parses the circuit text itself and
 * hard-codes its own gate table.
 *
 * Precision: complex128 (C99 double complex) for the exact simulator
 * ("JUQCS-E", Sec. 2), FP32 with explicit fmaf for the two-byte codec mirror.
 *
 * What each function follows:
 *   orc_apply_1q / orc_run      Eq. 1: every amplitude pair (a0,a1) that
 *                               differs only in bit t is replaced by U(a0,a1);
 *                               gates on k qubits act on the 2^k amplitudes
 *                               that differ only in those bits (Sec. 2, the
 *                               sparse matrix-vector view).
 *   orc_dense                   Sec. 2: an N-qubit gate as a 2^N x 2^N matrix
 *                               (identity on the untouched qubits), multiplied
 *                               out densely.  Brute force, n <= 8.
 *   orc_expect_pauli            Sec. 3: <sigma^alpha_i> for the validation
 *                               observable <Q_alpha(i)> = (1 - <sigma>)/2.
 *   orc_enc_*                   Sec. 1/3: the adaptive two-byte amplitude
 *                               code.  The paper does not give the format;
 *                               the reading implemented is: blocks of 256
 *                               amplitudes, block scale s = max(|re|,|im|),
 *                               int8 codes q = rint(x * fl(127/s)) clamped to
 *                               [-127,127], decode x = sign(q) * s * T[|q|]
 *                               with T[k] = fl(k/127).  Gates run in FP32 in a
 *                               fixed fmaf order, one decode-gate-encode per
 *                               gate.  Parity with the paper's own format is
 *                               therefore unpinned; the mirror is pinned by
 *                               properties (exact uniform state, round trip).
 *   orc_cut_amplitudes          Sec. 4, Eq. 2 and Eq. 3: every CZ between the
 *                               two partitions is replaced by a sum of
 *                               products of single-qubit operators; each term
 *                               s is simulated as two independent smaller
 *                               state vectors and <z|C|0> is the sum over s of
 *                               the products of their coefficients.
 *   orc_cut_amplitudes_multi    the same over P partitions (Sec. 4).
 *
 * Qubit j is bit j of the amplitude index (the paper leaves the order open).
 */
#include <complex.h>
#include <ctype.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

typedef double complex cplx;

enum { ORC_OK = 0, ORC_ERR_PARSE = 1, ORC_ERR_ARG = 2, ORC_ERR_MEM = 3, ORC_ERR_UNSUPPORTED = 4 };

static char orc_err[256];
const char *orc_last_error(void) { return orc_err; }

/* ------------------------------------------------------------------ */
/* Gate table (the reading of the gate set: principal square roots).   */
/* ------------------------------------------------------------------ */

typedef struct {
    int nq;          /* 1 or 2 */
    int q[2];        /* qubits; for 2-qubit gates local index = b(q0) + 2 b(q1) */
    cplx m[16];      /* 2x2 or 4x4 row-major */
} orc_gate;

static int one_qubit_matrix(const char *name, const double *p, int np, cplx u[4]) {
    const double r2 = 1.0 / sqrt(2.0);
    memset(u, 0, 4 * sizeof(cplx));
    if (!strcmp(name, "H")) { u[0] = r2; u[1] = r2; u[2] = r2; u[3] = -r2; }
    else if (!strcmp(name, "X")) { u[1] = 1; u[2] = 1; }
    else if (!strcmp(name, "Y")) { u[1] = -I; u[2] = I; }
    else if (!strcmp(name, "Z")) { u[0] = 1; u[3] = -1; }
    else if (!strcmp(name, "S")) { u[0] = 1; u[3] = I; }
    else if (!strcmp(name, "SDG")) { u[0] = 1; u[3] = -I; }
    else if (!strcmp(name, "T")) { u[0] = 1; u[3] = cexp(I * M_PI / 4); }
    else if (!strcmp(name, "TDG")) { u[0] = 1; u[3] = cexp(-I * M_PI / 4); }
    else if (!strcmp(name, "SX")) { u[0] = 0.5 * (1 + I); u[1] = 0.5 * (1 - I); u[2] = 0.5 * (1 - I); u[3] = 0.5 * (1 + I); }
    else if (!strcmp(name, "SXDG")) { u[0] = 0.5 * (1 - I); u[1] = 0.5 * (1 + I); u[2] = 0.5 * (1 + I); u[3] = 0.5 * (1 - I); }
    else if (!strcmp(name, "SY")) { u[0] = 0.5 * (1 + I); u[1] = 0.5 * (-1 - I); u[2] = 0.5 * (1 + I); u[3] = 0.5 * (1 + I); }
    else if (!strcmp(name, "SYDG")) { u[0] = 0.5 * (1 - I); u[1] = 0.5 * (1 - I); u[2] = 0.5 * (-1 + I); u[3] = 0.5 * (1 - I); }
    else if (!strcmp(name, "P")) { if (np != 1) return -1; u[0] = 1; u[3] = cexp(I * p[0]); }
    else if (!strcmp(name, "U")) {
        if (np != 8) return -1;
        for (int k = 0; k < 4; k++) u[k] = p[2 * k] + I * p[2 * k + 1];
    } else return -1;
    return 0;
}

static int two_qubit_matrix(const char *name, const double *p, int np, cplx m[16]) {
    memset(m, 0, 16 * sizeof(cplx));
    if (!strcmp(name, "CZ")) { m[0] = 1; m[5] = 1; m[10] = 1; m[15] = -1; }
    else if (!strcmp(name, "CP")) { if (np != 1) return -1; m[0] = 1; m[5] = 1; m[10] = 1; m[15] = cexp(I * p[0]); }
    else if (!strcmp(name, "CX")) { /* local index c + 2t: t flips where c = 1 */
        m[0 * 4 + 0] = 1; m[2 * 4 + 2] = 1; m[1 * 4 + 3] = 1; m[3 * 4 + 1] = 1; }
    else if (!strcmp(name, "SWAP")) { m[0] = 1; m[1 * 4 + 2] = 1; m[2 * 4 + 1] = 1; m[15] = 1; }
    else return -1;
    return 0;
}

/* Exported so the tests can compare the tables of the two sides. */
int orc_gate_matrix(const char *name, const double *params, int np, double *out /* 2*4 or 2*16 */) {
    cplx m[16];
    if (one_qubit_matrix(name, params, np, m) == 0) {
        for (int k = 0; k < 4; k++) { out[2 * k] = creal(m[k]); out[2 * k + 1] = cimag(m[k]); }
        return 1;
    }
    if (two_qubit_matrix(name, params, np, m) == 0) {
        for (int k = 0; k < 16; k++) { out[2 * k] = creal(m[k]); out[2 * k + 1] = cimag(m[k]); }
        return 2;
    }
    return -1;
}

/* ------------------------------------------------------------------ */
/* Circuit text parser.                                                */
/* ------------------------------------------------------------------ */

typedef struct {
    char name[8];
    int nq;
    int q[2];
    int np;
    double p[8];
} orc_instr;

typedef struct {
    int n;
    int count;
    orc_instr *v;
} orc_circuit;

static void circuit_free(orc_circuit *c) { free(c->v); c->v = NULL; c->count = 0; }

static int parse_circuit(const char *text, int n_expected, orc_circuit *out) {
    out->n = -1; out->count = 0; out->v = NULL;
    int cap = 0;
    const char *s = text;
    int lineno = 0;
    while (*s) {
        const char *e = strchr(s, '\n');
        size_t len = e ? (size_t)(e - s) : strlen(s);
        char line[512];
        lineno++;
        if (len >= sizeof line) { snprintf(orc_err, sizeof orc_err, "line %d too long", lineno); circuit_free(out); return ORC_ERR_PARSE; }
        memcpy(line, s, len); line[len] = 0;
        s = e ? e + 1 : s + len;
        char *hash = strchr(line, '#');
        if (hash) *hash = 0;
        char *tok[12]; int nt = 0;
        for (char *t = strtok(line, " \t\r"); t && nt < 12; t = strtok(NULL, " \t\r")) tok[nt++] = t;
        if (nt == 0) continue;
        if (!strcmp(tok[0], "qubits")) {
            if (nt != 2) { snprintf(orc_err, sizeof orc_err, "line %d: bad qubits line", lineno); circuit_free(out); return ORC_ERR_PARSE; }
            out->n = atoi(tok[1]);
            continue;
        }
        orc_instr in; memset(&in, 0, sizeof in);
        if (strlen(tok[0]) >= sizeof in.name) { snprintf(orc_err, sizeof orc_err, "line %d: unknown gate", lineno); circuit_free(out); return ORC_ERR_PARSE; }
        strcpy(in.name, tok[0]);
        int two = !strcmp(in.name, "CZ") || !strcmp(in.name, "CX") || !strcmp(in.name, "CP") || !strcmp(in.name, "SWAP");
        in.nq = two ? 2 : 1;
        if (nt < 1 + in.nq) { snprintf(orc_err, sizeof orc_err, "line %d: missing qubit", lineno); circuit_free(out); return ORC_ERR_PARSE; }
        for (int k = 0; k < in.nq; k++) in.q[k] = atoi(tok[1 + k]);
        in.np = nt - 1 - in.nq;
        if (in.np > 8) { snprintf(orc_err, sizeof orc_err, "line %d: too many params", lineno); circuit_free(out); return ORC_ERR_PARSE; }
        for (int k = 0; k < in.np; k++) in.p[k] = strtod(tok[1 + in.nq + k], NULL);
        cplx m[16];
        int ok = two ? two_qubit_matrix(in.name, in.p, in.np, m) : one_qubit_matrix(in.name, in.p, in.np, m);
        if (ok != 0) { snprintf(orc_err, sizeof orc_err, "line %d: unknown gate or bad params '%s'", lineno, in.name); circuit_free(out); return ORC_ERR_PARSE; }
        if (out->count == cap) {
            cap = cap ? 2 * cap : 64;
            orc_instr *nv = realloc(out->v, (size_t)cap * sizeof *nv);
            if (!nv) { circuit_free(out); return ORC_ERR_MEM; }
            out->v = nv;
        }
        out->v[out->count++] = in;
    }
    if (out->n < 0) out->n = n_expected;
    if (n_expected >= 0 && out->n != n_expected) { snprintf(orc_err, sizeof orc_err, "circuit has %d qubits, expected %d", out->n, n_expected); circuit_free(out); return ORC_ERR_ARG; }
    for (int g = 0; g < out->count; g++) {
        orc_instr *in = &out->v[g];
        for (int k = 0; k < in->nq; k++)
            if (in->q[k] < 0 || in->q[k] >= out->n) { snprintf(orc_err, sizeof orc_err, "gate %d: qubit %d out of range", g, in->q[k]); circuit_free(out); return ORC_ERR_ARG; }
        if (in->nq == 2 && in->q[0] == in->q[1]) { snprintf(orc_err, sizeof orc_err, "gate %d: repeated qubit", g); circuit_free(out); return ORC_ERR_ARG; }
    }
    return ORC_OK;
}

static void instr_gate(const orc_instr *in, orc_gate *g) {
    g->nq = in->nq; g->q[0] = in->q[0]; g->q[1] = in->q[1];
    if (in->nq == 1) one_qubit_matrix(in->name, in->p, in->np, g->m);
    else two_qubit_matrix(in->name, in->p, in->np, g->m);
}

/* ------------------------------------------------------------------ */
/* Exact simulator (complex128).                                       */
/* ------------------------------------------------------------------ */

/* Eq. 1 on qubit t: for every index i with bit t clear, (psi_i, psi_{i+2^t})
 * <- U (psi_i, psi_{i+2^t}). */
void orc_apply_1q(double *psi_d, int n, int t, const double *u_d) {
    cplx *psi = (cplx *)psi_d;
    cplx u[4];
    for (int k = 0; k < 4; k++) u[k] = u_d[2 * k] + I * u_d[2 * k + 1];
    uint64_t dim = (uint64_t)1 << n, bit = (uint64_t)1 << t;
    for (uint64_t i = 0; i < dim; i++) {
        if (i & bit) continue;
        cplx a0 = psi[i], a1 = psi[i | bit];
        psi[i] = u[0] * a0 + u[1] * a1;
        psi[i | bit] = u[2] * a0 + u[3] * a1;
    }
}

/* A k-qubit matrix (2^k x 2^k, row-major; local index bit j <-> qubits[j])
 * applied to the 2^k amplitudes that differ only in those qubits. */
int orc_apply_kq(double *psi_d, int n, int k, const int *qubits, const double *u_d) {
    if (k < 1 || k > 10) return ORC_ERR_ARG;
    cplx *psi = (cplx *)psi_d;
    uint64_t mask = 0;
    for (int j = 0; j < k; j++) {
        if (qubits[j] < 0 || qubits[j] >= n || (mask >> qubits[j] & 1)) return ORC_ERR_ARG;
        mask |= (uint64_t)1 << qubits[j];
    }
    int d = 1 << k;
    cplx *in = malloc(sizeof(cplx) * d), *outv = malloc(sizeof(cplx) * d);
    uint64_t *off = malloc(sizeof(uint64_t) * d);
    if (!in || !outv || !off) { free(in); free(outv); free(off); return ORC_ERR_MEM; }
    for (int l = 0; l < d; l++) {
        uint64_t o = 0;
        for (int j = 0; j < k; j++) if (l >> j & 1) o |= (uint64_t)1 << qubits[j];
        off[l] = o;
    }
    uint64_t dim = (uint64_t)1 << n;
    for (uint64_t i = 0; i < dim; i++) {
        if (i & mask) continue;
        for (int l = 0; l < d; l++) in[l] = psi[i | off[l]];
        for (int r = 0; r < d; r++) {
            cplx acc = 0;
            for (int c = 0; c < d; c++) acc += (u_d[2 * (r * d + c)] + I * u_d[2 * (r * d + c) + 1]) * in[c];
            outv[r] = acc;
        }
        for (int l = 0; l < d; l++) psi[i | off[l]] = outv[l];
    }
    free(in); free(outv); free(off);
    return ORC_OK;
}

static void apply_gate(cplx *psi, int n, const orc_gate *g) {
    double m[32];
    int d = g->nq == 1 ? 4 : 16;
    for (int k = 0; k < d; k++) { m[2 * k] = creal(g->m[k]); m[2 * k + 1] = cimag(g->m[k]); }
    if (g->nq == 1) orc_apply_1q((double *)psi, n, g->q[0], m);
    else orc_apply_kq((double *)psi, n, 2, g->q, m);
}

/* Apply every gate of the circuit text, in order, to psi (in place). */
int orc_run(const char *text, int n, double *psi) {
    orc_circuit c;
    int rc = parse_circuit(text, n, &c);
    if (rc) return rc;
    for (int g = 0; g < c.count; g++) {
        orc_gate gate;
        instr_gate(&c.v[g], &gate);
        apply_gate((cplx *)psi, n, &gate);
    }
    circuit_free(&c);
    return ORC_OK;
}

/* Number of gates in a circuit text (or a negative error code). */
int orc_count_gates(const char *text) {
    orc_circuit c;
    int rc = parse_circuit(text, -1, &c);
    if (rc) return -rc;
    int k = c.count;
    circuit_free(&c);
    return k;
}

/* Brute force: the full 2^n x 2^n unitary of the circuit.  Each gate's full
 * matrix has entry G[i][j] = g[loc(i)][loc(j)] when i and j agree on every
 * qubit the gate does not touch, else 0; the circuit matrix is the ordered
 * product, computed with plain triple loops. */
int orc_dense(const char *text, int n, double *out) {
    if (n < 1 || n > 8) return ORC_ERR_ARG;
    orc_circuit c;
    int rc = parse_circuit(text, n, &c);
    if (rc) return rc;
    size_t dim = (size_t)1 << n;
    cplx *M = calloc(dim * dim, sizeof(cplx)), *G = calloc(dim * dim, sizeof(cplx)), *T = calloc(dim * dim, sizeof(cplx));
    if (!M || !G || !T) { free(M); free(G); free(T); circuit_free(&c); return ORC_ERR_MEM; }
    for (size_t i = 0; i < dim; i++) M[i * dim + i] = 1;
    for (int g = 0; g < c.count; g++) {
        orc_gate gate;
        instr_gate(&c.v[g], &gate);
        size_t touched = 0;
        for (int k = 0; k < gate.nq; k++) touched |= (size_t)1 << gate.q[k];
        int d = 1 << gate.nq;
        for (size_t i = 0; i < dim; i++)
            for (size_t j = 0; j < dim; j++) {
                if ((i & ~touched) != (j & ~touched)) { G[i * dim + j] = 0; continue; }
                int li = 0, lj = 0;
                for (int k = 0; k < gate.nq; k++) {
                    li |= (int)((i >> gate.q[k]) & 1) << k;
                    lj |= (int)((j >> gate.q[k]) & 1) << k;
                }
                G[i * dim + j] = gate.m[li * d + lj];
            }
        for (size_t i = 0; i < dim; i++)
            for (size_t j = 0; j < dim; j++) {
                cplx acc = 0;
                for (size_t l = 0; l < dim; l++) acc += G[i * dim + l] * M[l * dim + j];
                T[i * dim + j] = acc;
            }
        cplx *sw = M; M = T; T = sw;
    }
    for (size_t k = 0; k < dim * dim; k++) { out[2 * k] = creal(M[k]); out[2 * k + 1] = cimag(M[k]); }
    free(M); free(G); free(T); circuit_free(&c);
    return ORC_OK;
}

/* sum_i |psi_i|^2 */
double orc_norm(const double *psi, int n) {
    uint64_t dim = (uint64_t)1 << n;
    double s = 0;
    for (uint64_t i = 0; i < dim; i++) s += psi[2 * i] * psi[2 * i] + psi[2 * i + 1] * psi[2 * i + 1];
    return s;
}

/* <psi| sigma^alpha_q |psi> for alpha = 0 (x), 1 (y), 2 (z), by applying the
 * Pauli matrix to a copy and taking the inner product (Sec. 3). */
int orc_expect_pauli(const double *psi_d, int n, int q, int alpha, double *out) {
    if (q < 0 || q >= n || alpha < 0 || alpha > 2) return ORC_ERR_ARG;
    uint64_t dim = (uint64_t)1 << n;
    cplx *phi = malloc(dim * sizeof(cplx));
    if (!phi) return ORC_ERR_MEM;
    memcpy(phi, psi_d, dim * sizeof(cplx));
    double sig[3][8] = {
        {0, 0, 1, 0, 1, 0, 0, 0},   /* x */
        {0, 0, 0, -1, 0, 1, 0, 0},  /* y */
        {1, 0, 0, 0, 0, 0, -1, 0},  /* z */
    };
    orc_apply_1q((double *)phi, n, q, sig[alpha]);
    const cplx *psi = (const cplx *)psi_d;
    cplx acc = 0;
    for (uint64_t i = 0; i < dim; i++) acc += conj(psi[i]) * phi[i];
    free(phi);
    *out = creal(acc);
    return ORC_OK;
}

/* ------------------------------------------------------------------ */
/* Two-byte codec mirror (FP32, bit-exact definition of the reading).  */
/* ------------------------------------------------------------------ */

#define ENC_BLOCK 256

/* T[k] = fl(k / 127) (IEEE single division, round to nearest). */
static float enc_table(int k) { return (float)k / 127.0f; }

static float enc_decode_one(int8_t q, float scale) {
    int a = q < 0 ? -q : q;
    float v = scale * enc_table(a);
    return q < 0 ? -v : v;
}

static int8_t enc_encode_one(float x, float inv) {
    float y = x * inv;               /* one rounded FP32 product */
    float r = rintf(y);              /* round half to even */
    if (r > 127.0f) r = 127.0f;
    if (r < -127.0f) r = -127.0f;
    return (int8_t)r;
}

/* Encode 2^n FP32 complex amplitudes (interleaved) into int8 codes
 * (interleaved re,im) and one FP32 scale per block of 256 amplitudes. */
int orc_enc_encode(const float *psi, int n, int8_t *codes, float *scales) {
    uint64_t dim = (uint64_t)1 << n;
    uint64_t nb = dim < ENC_BLOCK ? 1 : dim / ENC_BLOCK;
    uint64_t bsz = dim < ENC_BLOCK ? dim : ENC_BLOCK;
    for (uint64_t b = 0; b < nb; b++) {
        float s = 0.0f;
        for (uint64_t j = 0; j < 2 * bsz; j++) {
            float a = fabsf(psi[2 * b * bsz + j]);
            if (a > s) s = a;
        }
        scales[b] = s;
        if (s == 0.0f) {
            for (uint64_t j = 0; j < 2 * bsz; j++) codes[2 * b * bsz + j] = 0;
            continue;
        }
        float inv = 127.0f / s;
        for (uint64_t j = 0; j < 2 * bsz; j++) codes[2 * b * bsz + j] = enc_encode_one(psi[2 * b * bsz + j], inv);
    }
    return ORC_OK;
}

int orc_enc_decode(const int8_t *codes, const float *scales, int n, float *psi) {
    uint64_t dim = (uint64_t)1 << n;
    uint64_t bsz = dim < ENC_BLOCK ? dim : ENC_BLOCK;
    for (uint64_t i = 0; i < 2 * dim; i++) psi[i] = enc_decode_one(codes[i], scales[(i / 2) / bsz]);
    return ORC_OK;
}

/* The FP32 gate in the fixed evaluation order of the reading:
 *   re' = fma(u_r, a_r, fma(-u_i, a_i, fma(v_r, b_r, -(v_i * b_i))))
 *   im' = fma(u_r, a_i, fma(u_i, a_r, fma(v_r, b_i, v_i * b_r)))
 * for each output row (u, v) of the 2x2 matrix. */
static void enc_gate_pair(const float *u, float *a, float *b) {
    float ar = a[0], ai = a[1], br = b[0], bi = b[1];
    float r0 = fmaf(u[0], ar, fmaf(-u[1], ai, fmaf(u[2], br, -(u[3] * bi))));
    float i0 = fmaf(u[0], ai, fmaf(u[1], ar, fmaf(u[2], bi, u[3] * br)));
    float r1 = fmaf(u[4], ar, fmaf(-u[5], ai, fmaf(u[6], br, -(u[7] * bi))));
    float i1 = fmaf(u[4], ai, fmaf(u[5], ar, fmaf(u[6], bi, u[7] * br)));
    a[0] = r0; a[1] = i0; b[0] = r1; b[1] = i1;
}

/* One gate on the encoded state: decode everything, apply the FP32 gate to
 * every pair (bit t clear / set) whose control bit is 1 (control < 0: no
 * control), re-encode everything with fresh block scales. */
int orc_enc_apply_gate(int8_t *codes, float *scales, int n, int t, int control, const double *u_d) {
    if (t < 0 || t >= n || control >= n || control == t) return ORC_ERR_ARG;
    uint64_t dim = (uint64_t)1 << n;
    float *psi = malloc(2 * dim * sizeof(float));
    if (!psi) return ORC_ERR_MEM;
    orc_enc_decode(codes, scales, n, psi);
    float u[8];
    for (int k = 0; k < 8; k++) u[k] = (float)u_d[k];
    uint64_t bit = (uint64_t)1 << t;
    for (uint64_t i = 0; i < dim; i++) {
        if (i & bit) continue;
        if (control >= 0 && !((i >> control) & 1)) continue;
        enc_gate_pair(u, &psi[2 * i], &psi[2 * (i | bit)]);
    }
    orc_enc_encode(psi, n, codes, scales);
    free(psi);
    return ORC_OK;
}

/* Encoded run of a circuit text from |0...0>: each gate becomes one
 * (target, control, 2x2) update: CZ a b -> Z on b controlled by a,
 * CX c t -> X on t controlled by c, CP c t th -> P(th) on t controlled by c,
 * SWAP a b -> CX a b, CX b a, CX a b. */
int orc_enc_run(const char *text, int n, int8_t *codes, float *scales) {
    orc_circuit c;
    int rc = parse_circuit(text, n, &c);
    if (rc) return rc;
    for (int g = 0; g < c.count && rc == ORC_OK; g++) {
        orc_instr *in = &c.v[g];
        cplx u[4];
        double ud[8];
        if (in->nq == 1) {
            one_qubit_matrix(in->name, in->p, in->np, u);
            for (int k = 0; k < 4; k++) { ud[2 * k] = creal(u[k]); ud[2 * k + 1] = cimag(u[k]); }
            rc = orc_enc_apply_gate(codes, scales, n, in->q[0], -1, ud);
        } else if (!strcmp(in->name, "SWAP")) {
            double x[8] = {0, 0, 1, 0, 1, 0, 0, 0};
            int a = in->q[0], b = in->q[1];
            rc = orc_enc_apply_gate(codes, scales, n, b, a, x);
            if (!rc) rc = orc_enc_apply_gate(codes, scales, n, a, b, x);
            if (!rc) rc = orc_enc_apply_gate(codes, scales, n, b, a, x);
        } else {
            if (!strcmp(in->name, "CZ")) one_qubit_matrix("Z", NULL, 0, u);
            else if (!strcmp(in->name, "CX")) one_qubit_matrix("X", NULL, 0, u);
            else one_qubit_matrix("P", in->p, 1, u);
            for (int k = 0; k < 4; k++) { ud[2 * k] = creal(u[k]); ud[2 * k + 1] = cimag(u[k]); }
            rc = orc_enc_apply_gate(codes, scales, n, in->q[1], in->q[0], ud);
        }
    }
    circuit_free(&c);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Decomposition of entangling gates across two partitions (Sec. 4).   */
/* ------------------------------------------------------------------ */

/* Eq. 2: x solves cos(2x) = i; principal value from the complex arccosine. */
static cplx eq2_x(void) { return cacos(I) / 2.0; }

/* The single-qubit factor of the Eq. 2 term with sign s (+1 or -1):
 * exp(i sigma^z (x s - pi/4)) = diag(e^{i phi}, e^{-i phi}), phi = x s - pi/4. */
static void eq2_factor(int s, cplx d[2]) {
    cplx phi = eq2_x() * s - M_PI / 4;
    d[0] = cexp(I * phi);
    d[1] = cexp(-I * phi);
}

/* Exported for the tests: x, and the factors D_{+1}, D_{-1}. */
void orc_eq2_terms(double *x_out /*2*/, double *dplus /*4*/, double *dminus /*4*/) {
    cplx x = eq2_x(), d[2];
    x_out[0] = creal(x); x_out[1] = cimag(x);
    eq2_factor(+1, d);
    dplus[0] = creal(d[0]); dplus[1] = cimag(d[0]); dplus[2] = creal(d[1]); dplus[3] = cimag(d[1]);
    eq2_factor(-1, d);
    dminus[0] = creal(d[0]); dminus[1] = cimag(d[0]); dminus[2] = creal(d[1]); dminus[3] = cimag(d[1]);
}

typedef struct {
    int kind;       /* 0 gate, 1 branch op */
    orc_gate g;     /* kind 0: gate on local qubits */
    int q;          /* kind 1: local qubit */
    int cut;        /* kind 1: index of the decomposed gate */
    int role;       /* kind 1: 0 = partition A side, 1 = partition B side */
    double theta;   /* kind 1: phase of the decomposed controlled phase (pi for CZ) */
} half_op;

typedef struct { int count, cap; half_op *v; } half_prog;

static int prog_push(half_prog *p, half_op op) {
    if (p->count == p->cap) {
        p->cap = p->cap ? 2 * p->cap : 64;
        half_op *nv = realloc(p->v, (size_t)p->cap * sizeof *nv);
        if (!nv) return ORC_ERR_MEM;
        p->v = nv;
    }
    p->v[p->count++] = op;
    return ORC_OK;
}

/* Branch operator for term bit sb (0 <-> s=+1, 1 <-> s=-1) of one cut gate.
 * form 0 (projector): CP_ab(th) = P0(a) (x) 1 + P1(a) (x) diag(1, e^{i th});
 *   side A gets P_sb, side B gets 1 (sb=0) or diag(1, e^{i th}) (sb=1).
 * form 1 (Eq. 2, CZ only): both sides get exp(i sigma^z (x s - pi/4)). */
static void branch_diag(int form, int role, int sb, double theta, cplx d[2]) {
    if (form == 0) {
        if (role == 0) { d[0] = sb ? 0 : 1; d[1] = sb ? 1 : 0; }
        else { d[0] = 1; d[1] = sb ? cexp(I * theta) : 1; }
    } else {
        eq2_factor(sb ? -1 : +1, d);
    }
}

static void apply_diag1(cplx *psi, int n, int q, const cplx d[2]) {
    uint64_t dim = (uint64_t)1 << n;
    for (uint64_t i = 0; i < dim; i++) psi[i] *= d[(i >> q) & 1];
}

/* <z|C|0> for m bit strings z (Eq. 3): the qubits in maskA form partition
 * A, the rest partition B; every CZ or CP between A and B is decomposed
 * (CX between them is first rewritten as H CZ H on its target), and the sum
 * over all 2^S terms of <z_A|W_A(s)|0_A><z_B|W_B(s)|0_B> is returned as m
 * complex numbers.  form 0: projector decomposition (weight 1); form 1:
 * Eq. 2 (weight 1/2 per decomposed gate, CZ only).  n_cut_out, if not NULL,
 * receives S. */
static int cut_amplitudes_range(const char *text, int n, uint64_t maskA, int form, uint64_t s_lo, uint64_t s_step,
                                int64_t m, const uint64_t *z, double *out, int *n_cut_out);

int orc_cut_amplitudes(const char *text, int n, uint64_t maskA, int form,
                       int64_t m, const uint64_t *z, double *out, int *n_cut_out) {
    return cut_amplitudes_range(text, n, maskA, form, 0, 1, m, z, out, n_cut_out);
}

/* The part of the Eq. 3 sum over the terms s = part, part + 2^p, part + 2 * 2^p,
 * ... (the terms are independent, Sec. 4, so parts can be summed anywhere). */
int orc_cut_amplitudes_part(const char *text, int n, uint64_t maskA, int form, uint64_t part, int nparts_log2,
                            int64_t m, const uint64_t *z, double *out, int *n_cut_out) {
    if (nparts_log2 < 0 || nparts_log2 > 20 || (part >> nparts_log2)) return ORC_ERR_ARG;
    return cut_amplitudes_range(text, n, maskA, form, part, (uint64_t)1 << nparts_log2, m, z, out, n_cut_out);
}

static int cut_amplitudes_range(const char *text, int n, uint64_t maskA, int form, uint64_t s_lo, uint64_t s_step,
                                int64_t m, const uint64_t *z, double *out, int *n_cut_out) {
    if (form != 0 && form != 1) return ORC_ERR_ARG;
    orc_circuit c;
    int rc = parse_circuit(text, n, &c);
    if (rc) return rc;
    int loc[64], side[64], nA = 0, nB = 0;
    for (int q = 0; q < n; q++) {
        side[q] = (maskA >> q & 1) ? 0 : 1;
        loc[q] = side[q] == 0 ? nA++ : nB++;
    }
    if (nA == 0 || nB == 0 || nA > 28 || nB > 28) { circuit_free(&c); snprintf(orc_err, sizeof orc_err, "bad partition sizes %d/%d", nA, nB); return ORC_ERR_ARG; }
    half_prog prog[2] = {{0, 0, NULL}, {0, 0, NULL}};
    int S = 0;
    for (int g = 0; g < c.count && rc == ORC_OK; g++) {
        orc_instr *in = &c.v[g];
        orc_gate gate;
        instr_gate(in, &gate);
        if (in->nq == 1 || side[in->q[0]] == side[in->q[1]]) {
            half_op op; memset(&op, 0, sizeof op);
            op.kind = 0; op.g = gate;
            for (int k = 0; k < gate.nq; k++) op.g.q[k] = loc[in->q[k]];
            rc = prog_push(&prog[side[in->q[0]]], op);
            continue;
        }
        /* an entangling gate between the partitions */
        int a = in->q[0], b = in->q[1];
        double theta;
        int hq = -1;
        if (!strcmp(in->name, "CZ")) theta = M_PI;
        else if (!strcmp(in->name, "CP")) theta = in->p[0];
        else if (!strcmp(in->name, "CX")) { theta = M_PI; hq = b; }
        else { rc = ORC_ERR_UNSUPPORTED; snprintf(orc_err, sizeof orc_err, "cannot decompose %s across the cut", in->name); break; }
        if (form == 1 && fabs(theta - M_PI) > 0) { rc = ORC_ERR_UNSUPPORTED; snprintf(orc_err, sizeof orc_err, "Eq. 2 form decomposes CZ only"); break; }
        if (S >= 20) { rc = ORC_ERR_UNSUPPORTED; snprintf(orc_err, sizeof orc_err, "too many decomposed gates"); break; }
        half_op h; memset(&h, 0, sizeof h);
        if (hq >= 0) {
            h.kind = 0; h.g.nq = 1; h.g.q[0] = loc[hq];
            one_qubit_matrix("H", NULL, 0, h.g.m);
            rc = prog_push(&prog[side[hq]], h);
            if (rc) break;
        }
        int qa = side[a] == 0 ? a : b, qb = side[a] == 0 ? b : a;
        half_op opA; memset(&opA, 0, sizeof opA);
        opA.kind = 1; opA.q = loc[qa]; opA.cut = S; opA.role = 0; opA.theta = theta;
        half_op opB = opA; opB.q = loc[qb]; opB.role = 1;
        rc = prog_push(&prog[0], opA);
        if (!rc) rc = prog_push(&prog[1], opB);
        if (!rc && hq >= 0) rc = prog_push(&prog[side[hq]], h);
        S++;
    }
    circuit_free(&c);
    if (rc) { free(prog[0].v); free(prog[1].v); return rc; }
    if (n_cut_out) *n_cut_out = S;
    int nh[2] = {nA, nB};
    cplx *psi[2];
    psi[0] = malloc(((uint64_t)1 << nA) * sizeof(cplx));
    psi[1] = malloc(((uint64_t)1 << nB) * sizeof(cplx));
    uint64_t *zh[2];
    zh[0] = malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    zh[1] = malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
    cplx *acc = calloc((size_t)(m > 0 ? m : 1), sizeof(cplx));
    if (!psi[0] || !psi[1] || !zh[0] || !zh[1] || !acc) { rc = ORC_ERR_MEM; goto done; }
    for (int64_t j = 0; j < m; j++) {     /* split each z into z_A and z_B */
        uint64_t za = 0, zb = 0;
        for (int q = 0; q < n; q++) {
            uint64_t bitv = (z[j] >> q) & 1;
            if (side[q] == 0) za |= bitv << loc[q]; else zb |= bitv << loc[q];
        }
        zh[0][j] = za; zh[1][j] = zb;
    }
    double w = form == 1 ? ldexp(1.0, -S) : 1.0;
    for (uint64_t s = s_lo; s < ((uint64_t)1 << S); s += s_step) {
        for (int p = 0; p < 2; p++) {
            uint64_t dim = (uint64_t)1 << nh[p];
            memset(psi[p], 0, dim * sizeof(cplx));
            psi[p][0] = 1;
            for (int k = 0; k < prog[p].count; k++) {
                half_op *op = &prog[p].v[k];
                if (op->kind == 0) apply_gate(psi[p], nh[p], &op->g);
                else {
                    cplx d[2];
                    branch_diag(form, op->role, (int)((s >> op->cut) & 1), op->theta, d);
                    apply_diag1(psi[p], nh[p], op->q, d);
                }
            }
        }
        for (int64_t j = 0; j < m; j++) acc[j] += w * psi[0][zh[0][j]] * psi[1][zh[1][j]];
    }
    for (int64_t j = 0; j < m; j++) { out[2 * j] = creal(acc[j]); out[2 * j + 1] = cimag(acc[j]); }
done:
    free(psi[0]); free(psi[1]); free(zh[0]); free(zh[1]); free(acc);
    free(prog[0].v); free(prog[1].v);
    return rc;
}


/* <z|C|0> over P partitions (Sec. 4: the sum over s of products of P
 * circuits that each act on one partition).  part_of[q] is the partition of
 * qubit q; every CZ, CP or CX between two partitions is decomposed as in
 * orc_cut_amplitudes, the projector (or first Eq. 2 factor) on the
 * partition of the gate's first qubit.  Each term s is simulated as P
 * independent state vectors and the products of their coefficients are
 * summed (terms s = part mod 2^nparts_log2 only).  z: m bit strings of
 * nwords 64-bit words (qubit q is bit q % 64 of word q / 64). */
int orc_cut_amplitudes_multi(const char *text, int n, const unsigned char *part_of, int P, int form, uint64_t part,
                             int nparts_log2, int64_t m, const uint64_t *z, int nwords, double *out, int *n_cut_out) {
    enum { MAXP = 16, MAXQ = 128 };
    if (form != 0 && form != 1) return ORC_ERR_ARG;
    if (n < 2 || n > MAXQ || P < 2 || P > MAXP || nwords != (n + 63) / 64) return ORC_ERR_ARG;
    if (nparts_log2 < 0 || nparts_log2 > 20 || (part >> nparts_log2)) return ORC_ERR_ARG;
    int loc[MAXQ], side[MAXQ], np[MAXP] = {0};
    for (int q = 0; q < n; q++) {
        if (part_of[q] >= P) return ORC_ERR_ARG;
        side[q] = part_of[q];
        loc[q] = np[side[q]]++;
    }
    for (int p = 0; p < P; p++)
        if (np[p] == 0 || np[p] > 24) { snprintf(orc_err, sizeof orc_err, "partition %d has %d qubits", p, np[p]); return ORC_ERR_ARG; }
    orc_circuit c;
    int rc = parse_circuit(text, n, &c);
    if (rc) return rc;
    half_prog prog[MAXP];
    memset(prog, 0, sizeof prog);
    int S = 0;
    for (int g = 0; g < c.count && rc == ORC_OK; g++) {
        orc_instr *in = &c.v[g];
        orc_gate gate;
        instr_gate(in, &gate);
        if (in->nq == 1 || side[in->q[0]] == side[in->q[1]]) {
            half_op op; memset(&op, 0, sizeof op);
            op.kind = 0; op.g = gate;
            for (int k = 0; k < gate.nq; k++) op.g.q[k] = loc[in->q[k]];
            rc = prog_push(&prog[side[in->q[0]]], op);
            continue;
        }
        int a = in->q[0], b = in->q[1];
        double theta;
        int hq = -1;
        if (!strcmp(in->name, "CZ")) theta = M_PI;
        else if (!strcmp(in->name, "CP")) theta = in->p[0];
        else if (!strcmp(in->name, "CX")) { theta = M_PI; hq = b; }
        else { rc = ORC_ERR_UNSUPPORTED; snprintf(orc_err, sizeof orc_err, "cannot decompose %s across partitions", in->name); break; }
        if (form == 1 && fabs(theta - M_PI) > 0) { rc = ORC_ERR_UNSUPPORTED; snprintf(orc_err, sizeof orc_err, "Eq. 2 form decomposes CZ only"); break; }
        if (S >= 20) { rc = ORC_ERR_UNSUPPORTED; snprintf(orc_err, sizeof orc_err, "too many decomposed gates"); break; }
        half_op h; memset(&h, 0, sizeof h);
        if (hq >= 0) {
            h.kind = 0; h.g.nq = 1; h.g.q[0] = loc[hq];
            one_qubit_matrix("H", NULL, 0, h.g.m);
            rc = prog_push(&prog[side[hq]], h);
            if (rc) break;
        }
        half_op opA; memset(&opA, 0, sizeof opA);
        opA.kind = 1; opA.q = loc[a]; opA.cut = S; opA.role = 0; opA.theta = theta;
        half_op opB = opA; opB.q = loc[b]; opB.role = 1;
        rc = prog_push(&prog[side[a]], opA);
        if (!rc) rc = prog_push(&prog[side[b]], opB);
        if (!rc && hq >= 0) rc = prog_push(&prog[side[hq]], h);
        S++;
    }
    circuit_free(&c);
    cplx *psi[MAXP] = {0};
    uint64_t *zp[MAXP] = {0};
    cplx *acc = NULL;
    if (rc) goto done;
    if (n_cut_out) *n_cut_out = S;
    for (int p = 0; p < P; p++) {
        psi[p] = malloc(((uint64_t)1 << np[p]) * sizeof(cplx));
        zp[p] = malloc((size_t)(m > 0 ? m : 1) * sizeof(uint64_t));
        if (!psi[p] || !zp[p]) { rc = ORC_ERR_MEM; goto done; }
    }
    acc = calloc((size_t)(m > 0 ? m : 1), sizeof(cplx));
    if (!acc) { rc = ORC_ERR_MEM; goto done; }
    for (int64_t j = 0; j < m; j++) {  /* each z split into its partitions' indices */
        for (int p = 0; p < P; p++) zp[p][j] = 0;
        for (int q = 0; q < n; q++) {
            uint64_t bitv = (z[j * nwords + q / 64] >> (q % 64)) & 1;
            zp[side[q]][j] |= bitv << loc[q];
        }
    }
    double w = form == 1 ? ldexp(1.0, -S) : 1.0;
    for (uint64_t s = part; s < ((uint64_t)1 << S); s += (uint64_t)1 << nparts_log2) {
        for (int p = 0; p < P; p++) {
            uint64_t dim = (uint64_t)1 << np[p];
            memset(psi[p], 0, dim * sizeof(cplx));
            psi[p][0] = 1;
            for (int k = 0; k < prog[p].count; k++) {
                half_op *op = &prog[p].v[k];
                if (op->kind == 0) apply_gate(psi[p], np[p], &op->g);
                else {
                    cplx d[2];
                    branch_diag(form, op->role, (int)((s >> op->cut) & 1), op->theta, d);
                    apply_diag1(psi[p], np[p], op->q, d);
                }
            }
        }
        for (int64_t j = 0; j < m; j++) {
            cplx t = w;
            for (int p = 0; p < P; p++) t *= psi[p][zp[p][j]];
            acc[j] += t;
        }
    }
    for (int64_t j = 0; j < m; j++) { out[2 * j] = creal(acc[j]); out[2 * j + 1] = cimag(acc[j]); }
done:
    for (int p = 0; p < P; p++) { free(psi[p]); free(zp[p]); free(prog[p].v); }
    free(acc);
    return rc;
}
