/*
 * hqc_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, obviously correct CPU implementation of HQC.PKE key
 * generation, encryption and decryption as the OptHQC paper (arXiv
 * 2512.12904) states them, used only by tests/, by the smoke check and by
 * the CPU-baseline leg of bench.py.  It shares no code, table, header or
 * constant generator with the CUDA library: every value below is derived
 * here from the paper's definitions.
 *
 * Sources (paper sections / algorithms / equations / tables):
 *   Table I          parameter sets HQC-1/3/5 (n, w, w_e = w_r, RS and RM codes)
 *   Algorithm 1      HQC.PKE.Encrypt: u = r1 + h*r2, v = mG + s*r2 + e
 *   Algorithm 2      HQC.PKE.Decrypt: m' = C.Decode(v - u*y)  (see reading A1)
 *   Algorithm 3      HQC.KEM.KeyGen core: s = x + h*y
 *   Eq. 1 (Sec. III-B) sparse x dense product as the XOR of rotations
 *   Sec. II-A        concatenated code: shortened RS outer code, duplicated
 *                    RM(1,7) inner code; byte-parallel RM decoder
 *   Sec. III-D       RS syndromes S_i = sum_j c_j alpha^{i j}, i = 1..2*delta
 *
 * Readings where the paper is silent (the CUDA path follows the same list):
 *   A1 decrypt uses v - u*y (the paper prints u*s; y is the secret operand
 *      that cancels h: v - u*y = mG + x*r2 - r1*y + e).
 *   A2 v holds only the first n1*n2 bits; u*y is truncated the same way.
 *   A3 GF(2^8) = GF(2)[x]/(x^8+x^4+x^3+x^2+1), alpha = x.
 *   A4 RS generator g(x) = prod_{i=1}^{2 delta} (x - alpha^i).
 *   A5 bit i of a vector is bit (i mod 64) of 64-bit word i/64.
 *   A6 RS codeword c = (parity bytes || message bytes), c_j the x^j
 *      coefficient, parity = x^{n1-k} m(x) mod g(x).
 *   A7 RM(1,7): codeword bit i of byte a + 128 b is b XOR parity(a AND i);
 *      symbol j occupies bits [j n2, (j+1) n2) as mult copies of 128 bits.
 *   A8 RM decode: argmax over a of |F(a)|, ties to the smallest a,
 *      b = [F(a*) < 0].
 *   A9 textbook Berlekamp-Massey, exactly 2 delta iterations.
 *   A10 position j in error iff Lambda(alpha^{-j}) = 0, j in [0, n1).
 *   A11 Forney with first root alpha^1: e_j = Omega(alpha^{-j}) /
 *      Lambda'(alpha^{-j}), Omega = S Lambda mod x^{2 delta}; x/0 := 0.
 *   A12 nothing special happens beyond delta errors: A9-A11 applied
 *      literally define the output.  That output is "parity unpinned"
 *      against anything outside this file.
 *
 * Everything is unpacked (one byte per bit / per field element) and
 * computed straight from the definitions.  Nothing here is constant-time.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ */
/* Table I, written down as printed: N, w, w_e = w_r, RS [n1, k, d_RS],  */
/* RM [n2, 8, d_RM].  delta and the duplication factor are derived.     */
/* ------------------------------------------------------------------ */
typedef struct {
    int level, n, w, we, rs_n1, rs_k, rs_d, rm_n2, rm_k, rm_d;
} table1_row;

static const table1_row TABLE1[3] = {
    {1, 17669,  66,  75, 46, 16, 31, 384, 8, 192},
    {3, 35851, 100, 114, 56, 24, 33, 640, 8, 320},
    {5, 57637, 131, 149, 90, 32, 59, 640, 8, 320},
};

typedef struct {
    int n, w, wr, we, n1, k, delta, n2, mult;
} oparams;

static int get_params(int level, oparams *p)
{
    for (int i = 0; i < 3; i++) {
        if (TABLE1[i].level != level) continue;
        const table1_row *t = &TABLE1[i];
        p->n = t->n;
        p->w = t->w;
        p->wr = t->we;          /* Table I: w_e = w_r */
        p->we = t->we;
        p->n1 = t->rs_n1;
        p->k = t->rs_k;
        p->delta = (t->rs_d - 1) / 2;       /* RS corrects (d-1)/2 symbols */
        p->n2 = t->rm_n2;
        p->mult = t->rm_d / 64;             /* RM(1,7) has d = 64; copies add up */
        return 0;
    }
    return -1;
}

/* Exported for the parameter pin test: fills
 * [n, w, wr, we, n1, k, delta, n2, mult]. */
int oracle_params(int level, int32_t *out9)
{
    oparams p;
    if (get_params(level, &p)) return -1;
    int32_t v[9] = {p.n, p.w, p.wr, p.we, p.n1, p.k, p.delta, p.n2, p.mult};
    memcpy(out9, v, sizeof v);
    return 0;
}

/* ------------------------------------------------------------------ */
/* GF(2^8) (reading A3)                                                 */
/* ------------------------------------------------------------------ */
#define GF_POLY 0x11D   /* x^8 + x^4 + x^3 + x^2 + 1 */

/* Carry-less schoolbook product, then reduction by the modulus. */
uint8_t oracle_gf_mul(uint8_t a, uint8_t b)
{
    unsigned prod = 0;
    for (int i = 0; i < 8; i++)
        if ((b >> i) & 1) prod ^= (unsigned)a << i;
    for (int d = 14; d >= 8; d--)
        if ((prod >> d) & 1) prod ^= (unsigned)GF_POLY << (d - 8);
    return (uint8_t)prod;
}

/* a^e by repeated multiplication (e >= 0). */
static uint8_t gf_pow(uint8_t a, int e)
{
    uint8_t r = 1;
    for (int i = 0; i < e; i++) r = oracle_gf_mul(r, a);
    return r;
}

/* alpha^e for any integer e (alpha has order 255). */
static uint8_t gf_alpha(int e)
{
    e %= 255;
    if (e < 0) e += 255;
    return gf_pow(2, e);
}

/* Multiplicative inverse by exhaustive search; 0 maps to 0 (reading A11). */
static uint8_t gf_inv(uint8_t a)
{
    if (a == 0) return 0;
    for (int b = 1; b < 256; b++)
        if (oracle_gf_mul(a, (uint8_t)b) == 1) return (uint8_t)b;
    return 0; /* unreachable in a field */
}

/* ------------------------------------------------------------------ */
/* Reed-Solomon over GF(2^8), generic (n1, k) so tests can use tiny     */
/* codes; delta = (n1 - k) / 2.                                         */
/* ------------------------------------------------------------------ */

/* g(x) = prod_{i=1}^{2 delta} (x + alpha^i), coefficients g[0..2 delta]
 * (reading A4). */
int oracle_rs_generator(int n1, int k, uint8_t *g)
{
    int nr = n1 - k;
    if (nr <= 0 || nr > 254) return -1;
    memset(g, 0, (size_t)nr + 1);
    g[0] = 1;
    for (int i = 1; i <= nr; i++) {
        uint8_t root = gf_alpha(i);
        /* multiply the current polynomial (degree i-1) by (x + root) */
        for (int d = i; d >= 0; d--) {
            uint8_t shifted = (d > 0) ? g[d - 1] : 0;  /* x * g */
            g[d] = shifted ^ oracle_gf_mul(g[d], root); /* + root * g */
        }
    }
    return 0;
}

/* Systematic encoding (reading A6): c = parity || m, parity = the
 * remainder of x^{n1-k} m(x) divided by g(x), by plain long division. */
int oracle_rs_encode(int n1, int k, const uint8_t *m, uint8_t *c)
{
    int nr = n1 - k;
    uint8_t g[256];
    uint8_t rem[256];
    if (oracle_rs_generator(n1, k, g)) return -1;
    memset(rem, 0, sizeof rem);
    for (int i = 0; i < k; i++) rem[nr + i] = m[i];
    for (int d = n1 - 1; d >= nr; d--) {
        uint8_t coef = rem[d];
        if (!coef) continue;
        for (int i = 0; i <= nr; i++)
            rem[d - nr + i] ^= oracle_gf_mul(coef, g[i]);
    }
    for (int j = 0; j < nr; j++) c[j] = rem[j];
    for (int i = 0; i < k; i++) c[nr + i] = m[i];
    return 0;
}

/* S_i = sum_{j=0}^{n1-1} r_j alpha^{i j}, i = 1..2 delta (Sec. III-D).
 * S[i-1] holds S_i. */
int oracle_rs_syndromes(int n1, int k, const uint8_t *r, uint8_t *S)
{
    int nr = n1 - k;
    for (int i = 1; i <= nr; i++) {
        uint8_t acc = 0;
        for (int j = 0; j < n1; j++)
            acc ^= oracle_gf_mul(r[j], gf_alpha(i * j));
        S[i - 1] = acc;
    }
    return 0;
}

/* Evaluate a polynomial with ncoef coefficients at point x. */
static uint8_t poly_eval(const uint8_t *p, int ncoef, uint8_t x)
{
    uint8_t acc = 0;
    for (int i = 0; i < ncoef; i++)
        acc ^= oracle_gf_mul(p[i], gf_pow(x, i));
    return acc;
}

/*
 * Full RS decode of the received word r (reading A9-A11).
 *   S[2 delta]          syndromes S_1..S_{2 delta}
 *   lam[2 delta + 1]    error-locator Lambda_0..Lambda_{2 delta}
 *   L_out               final LFSR length of Berlekamp-Massey
 *   errmask[n1]         1 where Lambda(alpha^{-j}) = 0
 *   errval[n1]          Forney value at flagged positions, 0 elsewhere
 *   cw[n1]              r XOR errval
 *   flag_out            1 if L > delta or the number of roots found != L
 * Any output pointer may be NULL.
 */
int oracle_rs_decode(int n1, int k, const uint8_t *r, uint8_t *S_out,
                     uint8_t *lam_out, int32_t *L_out, uint8_t *errmask,
                     uint8_t *errval, uint8_t *cw, int32_t *flag_out)
{
    int nr = n1 - k;           /* = 2 delta */
    int cap = nr + 1;          /* Lambda and B hold 2 delta + 1 coefficients */
    uint8_t S[256], lam[256], B[256], T[256], omega[256];
    if (nr <= 0 || nr > 254 || n1 > 255) return -1;
    oracle_rs_syndromes(n1, k, r, S);

    /* Berlekamp-Massey, textbook form, exactly 2 delta iterations (A9). */
    memset(lam, 0, sizeof lam);
    memset(B, 0, sizeof B);
    lam[0] = 1;
    B[0] = 1;
    int L = 0, m = 1;
    uint8_t b = 1;
    for (int rr = 0; rr < nr; rr++) {
        /* discrepancy d = sum_{i=0}^{L} Lambda_i S_{r+1-i} */
        uint8_t d = 0;
        for (int i = 0; i <= L; i++)
            if (rr + 1 - i >= 1) d ^= oracle_gf_mul(lam[i], S[rr - i]);
        if (d == 0) {
            m += 1;
        } else {
            uint8_t coef = oracle_gf_mul(d, gf_inv(b));
            if (2 * L <= rr) {
                memcpy(T, lam, sizeof T);
                for (int i = 0; i < cap; i++)
                    if (i - m >= 0) lam[i] ^= oracle_gf_mul(coef, B[i - m]);
                L = rr + 1 - L;
                memcpy(B, T, sizeof B);
                b = d;
                m = 1;
            } else {
                for (int i = 0; i < cap; i++)
                    if (i - m >= 0) lam[i] ^= oracle_gf_mul(coef, B[i - m]);
                m += 1;
            }
        }
    }

    /* Omega(x) = S(x) Lambda(x) mod x^{2 delta}, S(x) = sum S_{i+1} x^i. */
    memset(omega, 0, sizeof omega);
    for (int a = 0; a < nr; a++)
        for (int c = 0; c < cap; c++)
            if (a + c < nr) omega[a + c] ^= oracle_gf_mul(S[a], lam[c]);

    /* Formal derivative: only odd-degree terms survive in characteristic 2. */
    uint8_t dlam[256];
    memset(dlam, 0, sizeof dlam);
    for (int i = 1; i < cap; i += 2) dlam[i - 1] = lam[i];

    int roots = 0;
    for (int j = 0; j < n1; j++) {
        uint8_t xinv = gf_alpha(-j);
        int is_root = poly_eval(lam, cap, xinv) == 0;
        uint8_t ev = 0;
        if (is_root) {
            uint8_t num = poly_eval(omega, nr, xinv);
            uint8_t den = poly_eval(dlam, cap, xinv);
            ev = (den == 0) ? 0 : oracle_gf_mul(num, gf_inv(den));
            roots++;
        }
        if (errmask) errmask[j] = (uint8_t)is_root;
        if (errval) errval[j] = ev;
        if (cw) cw[j] = r[j] ^ ev;
    }
    if (S_out) memcpy(S_out, S, (size_t)nr);
    if (lam_out) memcpy(lam_out, lam, (size_t)cap);
    if (L_out) *L_out = L;
    if (flag_out) *flag_out = (L > nr / 2) || (roots != L);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Reed-Muller RM(1,7), duplicated (reading A7, A8)                      */
/* ------------------------------------------------------------------ */
static int parity7(int x)
{
    int p = 0;
    for (int i = 0; i < 7; i++) p ^= (x >> i) & 1;
    return p;
}

/* bits[i] for i in [0,128) of the codeword of one byte. */
void oracle_rm_encode_byte(uint8_t byte, uint8_t *bits)
{
    int a = byte & 127, b = byte >> 7;
    for (int i = 0; i < 128; i++) bits[i] = (uint8_t)(b ^ parity7(a & i));
}

/* F(a) = sum_i s_i (-1)^{parity(a & i)} for a in [0,128), where
 * s_i = sum over the mult copies of (1 - 2 bit), straight from the
 * definition (no fast transform). */
void oracle_rm_transform(int mult, const uint8_t *bits, int32_t *F)
{
    int s[128];
    for (int i = 0; i < 128; i++) {
        s[i] = 0;
        for (int c = 0; c < mult; c++) s[i] += 1 - 2 * bits[128 * c + i];
    }
    for (int a = 0; a < 128; a++) {
        int acc = 0;
        for (int i = 0; i < 128; i++) acc += parity7(a & i) ? -s[i] : s[i];
        F[a] = acc;
    }
}

/* Byte decoded from one block of 128*mult received bits (reading A8). */
uint8_t oracle_rm_decode_block(int mult, const uint8_t *bits)
{
    int32_t F[128];
    oracle_rm_transform(mult, bits, F);
    int best = 0, best_abs = -1;
    for (int a = 0; a < 128; a++) {
        int v = F[a] < 0 ? -F[a] : F[a];
        if (v > best_abs) { best_abs = v; best = a; }   /* strict: smallest a wins ties */
    }
    return (uint8_t)(best + (F[best] < 0 ? 128 : 0));
}

/* ------------------------------------------------------------------ */
/* Ring GF(2)[x]/(x^n - 1), unpacked bits                               */
/* ------------------------------------------------------------------ */

/* Eq. 1: a1 * a2 mod (x^n - 1) = XOR over i in Supp(a1) of x^i * a2.
 * x^p * a2 has coefficient a2[(j - p) mod n] at x^j.  Entries p >= n
 * contribute nothing (library convention for malformed supports). */
void oracle_ring_mul_sparse(int n, const uint8_t *a2, const uint32_t *supp,
                            int wt, uint8_t *out)
{
    memset(out, 0, (size_t)n);
    for (int t = 0; t < wt; t++) {
        uint32_t p = supp[t];
        if (p >= (uint32_t)n) continue;
        for (int j = (int)p; j < n; j++) out[j] ^= a2[j - (int)p];
        for (int j = 0; j < (int)p; j++) out[j] ^= a2[j - (int)p + n];
    }
}

static void unpack_bits(const uint64_t *words, int nbits, uint8_t *bits)
{
    for (int i = 0; i < nbits; i++) bits[i] = (uint8_t)((words[i / 64] >> (i % 64)) & 1);
}

static void pack_bits(const uint8_t *bits, int nbits, uint64_t *words, int nwords)
{
    memset(words, 0, (size_t)nwords * 8);
    for (int i = 0; i < nbits; i++)
        if (bits[i]) words[i / 64] |= (uint64_t)1 << (i % 64);
}

/* Packed-word convenience wrapper for tests: out = a1 * a2 with a1 given
 * by its support, a2 and out as ceil(n/64) words. */
void oracle_ring_mul_packed(int n, const uint64_t *a2, const uint32_t *supp,
                            int wt, uint64_t *out)
{
    uint8_t *a = malloc((size_t)n), *o = malloc((size_t)n);
    unpack_bits(a2, n, a);
    oracle_ring_mul_sparse(n, a, supp, wt, o);
    pack_bits(o, n, out, (n + 63) / 64);
    free(a);
    free(o);
}

/* ------------------------------------------------------------------ */
/* Concatenated code C.Encode (Sec. II-A): RS encode, then each symbol   */
/* RM-encoded and duplicated mult times.  bits has n1*n2 entries.        */
/* ------------------------------------------------------------------ */
static void concat_encode(const oparams *p, const uint8_t *m, uint8_t *bits)
{
    uint8_t c[256], cwbits[128];
    oracle_rs_encode(p->n1, p->k, m, c);
    for (int j = 0; j < p->n1; j++) {
        oracle_rm_encode_byte(c[j], cwbits);
        for (int r = 0; r < p->mult; r++)
            for (int i = 0; i < 128; i++)
                bits[j * p->n2 + 128 * r + i] = cwbits[i];
    }
}

/* ------------------------------------------------------------------ */
/* PKE                                                                  */
/* ------------------------------------------------------------------ */
static int wu_pitch(const oparams *p) { int w = (p->n + 63) / 64; return w + (w & 1); }
static int wv(const oparams *p) { return (p->n1 * p->n2 + 63) / 64; }

/* Algorithm 3 core: s = x + h*y.  h, s: wu_pitch words (padding zero). */
static void keygen_one(const oparams *p, const uint64_t *h, const uint32_t *x,
                       const uint32_t *y, uint64_t *s)
{
    int n = p->n;
    uint8_t *hb = malloc((size_t)n), *sb = malloc((size_t)n);
    unpack_bits(h, n, hb);
    oracle_ring_mul_sparse(n, hb, y, p->w, sb);
    for (int t = 0; t < p->w; t++)
        if (x[t] < (uint32_t)n) sb[x[t]] ^= 1;
    pack_bits(sb, n, s, wu_pitch(p));
    free(hb);
    free(sb);
}

/* Algorithm 1: u = r1 + h*r2, v = first n1*n2 bits of mG + s*r2 + e. */
static void encrypt_one(const oparams *p, const uint64_t *h, const uint64_t *s,
                        const uint8_t *m, const uint32_t *r1, const uint32_t *r2,
                        const uint32_t *e, uint64_t *u, uint64_t *v)
{
    int n = p->n, nv = p->n1 * p->n2;
    uint8_t *hb = malloc((size_t)n), *sb = malloc((size_t)n);
    uint8_t *ub = malloc((size_t)n), *t = malloc((size_t)n);
    uint8_t *mg = malloc((size_t)nv);
    unpack_bits(h, n, hb);
    unpack_bits(s, n, sb);
    oracle_ring_mul_sparse(n, hb, r2, p->wr, ub);
    for (int i = 0; i < p->wr; i++)
        if (r1[i] < (uint32_t)n) ub[r1[i]] ^= 1;
    pack_bits(ub, n, u, wu_pitch(p));

    oracle_ring_mul_sparse(n, sb, r2, p->wr, t);
    for (int i = 0; i < p->we; i++)
        if (e[i] < (uint32_t)n) t[e[i]] ^= 1;
    concat_encode(p, m, mg);
    for (int i = 0; i < nv; i++) mg[i] ^= t[i];
    pack_bits(mg, nv, v, wv(p));
    free(hb); free(sb); free(ub); free(t); free(mg);
}

/* Algorithm 2 with reading A1, every intermediate kept. */
typedef struct {
    uint64_t *t, *w;            /* wv words each */
    uint8_t *r;                 /* n1 */
    uint8_t *S;                 /* 2 delta */
    uint8_t *lam;               /* 2 delta + 1 */
    int32_t *L;
    uint8_t *errmask, *errval, *cw;  /* n1 each */
    uint8_t *m;                 /* k */
    int32_t *flag;
} dump_ptrs;

static void decrypt_one(const oparams *p, const uint64_t *u, const uint64_t *v,
                        const uint32_t *y, const dump_ptrs *d)
{
    int n = p->n, nv = p->n1 * p->n2;
    uint8_t *ub = malloc((size_t)n), *prod = malloc((size_t)n);
    uint8_t *wb = malloc((size_t)nv);
    uint8_t r[256], cw[256];
    unpack_bits(u, n, ub);                 /* bits >= n of u are ignored */
    oracle_ring_mul_sparse(n, ub, y, p->w, prod);
    if (d->t) pack_bits(prod, nv, d->t, wv(p));
    unpack_bits(v, nv, wb);
    for (int i = 0; i < nv; i++) wb[i] ^= prod[i];   /* v - u*y, truncated */
    if (d->w) pack_bits(wb, nv, d->w, wv(p));
    for (int j = 0; j < p->n1; j++)
        r[j] = oracle_rm_decode_block(p->mult, wb + (size_t)j * p->n2);
    if (d->r) memcpy(d->r, r, (size_t)p->n1);
    oracle_rs_decode(p->n1, p->k, r, d->S, d->lam, d->L, d->errmask, d->errval,
                     cw, d->flag);
    if (d->cw) memcpy(d->cw, cw, (size_t)p->n1);
    if (d->m) memcpy(d->m, cw + (p->n1 - p->k), (size_t)p->k);
    free(ub); free(prod); free(wb);
}

/* ------------------------------------------------------------------ */
/* Batch entry points, threaded over independent items (static split). */
/* ------------------------------------------------------------------ */
typedef struct {
    int kind;                   /* 0 keygen, 1 encrypt, 2 decrypt */
    oparams p;
    int64_t begin, end;
    const uint64_t *h, *s, *u, *v;
    const uint32_t *x, *y, *r1, *r2, *e;
    const int32_t *key_idx;
    const uint8_t *m;
    uint64_t *s_out, *u_out, *v_out;
    uint8_t *m_out;
} job;

static void *run_job(void *arg)
{
    job *J = arg;
    const oparams *p = &J->p;
    int wp = wu_pitch(p), nvw = wv(p);
    for (int64_t i = J->begin; i < J->end; i++) {
        if (J->kind == 0) {
            keygen_one(p, J->h + i * wp, J->x + i * p->w, J->y + i * p->w, J->s_out + i * wp);
        } else if (J->kind == 1) {
            int64_t key = J->key_idx[i];
            encrypt_one(p, J->h + key * wp, J->s + key * wp, J->m + i * p->k,
                        J->r1 + i * p->wr, J->r2 + i * p->wr, J->e + i * p->we,
                        J->u_out + i * wp, J->v_out + i * nvw);
        } else {
            dump_ptrs d;
            memset(&d, 0, sizeof d);
            d.m = J->m_out + i * p->k;
            decrypt_one(p, J->u + i * wp, J->v + i * nvw, J->y + i * p->w, &d);
        }
    }
    return NULL;
}

static int run_batch(job proto, int64_t count, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 512) nthreads = 512;
    if (count < nthreads) nthreads = count > 0 ? (int)count : 1;
    pthread_t th[512];
    job jobs[512];
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = proto;
        jobs[t].begin = count * t / nthreads;
        jobs[t].end = count * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, run_job, &jobs[t]);
    run_job(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    return 0;
}

/* h, s_out: [nkeys][wu_pitch]; x, y: [nkeys][w]. */
int oracle_keygen_batch(int level, int64_t nkeys, const uint64_t *h,
                        const uint32_t *x, const uint32_t *y, uint64_t *s_out,
                        int nthreads)
{
    job J;
    memset(&J, 0, sizeof J);
    if (get_params(level, &J.p)) return -1;
    J.kind = 0; J.h = h; J.x = x; J.y = y; J.s_out = s_out;
    return run_batch(J, nkeys, nthreads);
}

/* h, s: [nkeys][wu_pitch]; key_idx[count]; m: [count][k];
 * r1, r2: [count][wr]; e: [count][we]; u_out: [count][wu_pitch];
 * v_out: [count][wv]. */
int oracle_encrypt_batch(int level, int64_t count, const uint64_t *h,
                         const uint64_t *s, const int32_t *key_idx,
                         const uint8_t *m, const uint32_t *r1,
                         const uint32_t *r2, const uint32_t *e,
                         uint64_t *u_out, uint64_t *v_out, int nthreads)
{
    job J;
    memset(&J, 0, sizeof J);
    if (get_params(level, &J.p)) return -1;
    J.kind = 1; J.h = h; J.s = s; J.key_idx = key_idx; J.m = m;
    J.r1 = r1; J.r2 = r2; J.e = e; J.u_out = u_out; J.v_out = v_out;
    return run_batch(J, count, nthreads);
}

/* u: [count][wu_pitch]; v: [count][wv]; y: [count][w] (literal supports);
 * m_out: [count][k]. */
int oracle_decrypt_batch(int level, int64_t count, const uint64_t *u,
                         const uint64_t *v, const uint32_t *y, uint8_t *m_out,
                         int nthreads)
{
    job J;
    memset(&J, 0, sizeof J);
    if (get_params(level, &J.p)) return -1;
    J.kind = 2; J.u = u; J.v = v; J.y = y; J.m_out = m_out;
    return run_batch(J, count, nthreads);
}

/* One ciphertext with every intermediate of Algorithm 2. */
int oracle_decrypt_dump(int level, const uint64_t *u, const uint64_t *v,
                        const uint32_t *y, uint64_t *t, uint64_t *w, uint8_t *r,
                        uint8_t *S, uint8_t *lam, int32_t *L, uint8_t *errmask,
                        uint8_t *errval, uint8_t *cw, uint8_t *m, int32_t *flag)
{
    oparams p;
    if (get_params(level, &p)) return -1;
    dump_ptrs d = {t, w, r, S, lam, L, errmask, errval, cw, m, flag};
    decrypt_one(&p, u, v, y, &d);
    return 0;
}

/* C.Encode of one message into n1*n2 packed bits (wv words), for tests. */
int oracle_concat_encode(int level, const uint8_t *m, uint64_t *out)
{
    oparams p;
    if (get_params(level, &p)) return -1;
    int nv = p.n1 * p.n2;
    uint8_t *bits = malloc((size_t)nv);
    concat_encode(&p, m, bits);
    pack_bits(bits, nv, out, wv(&p));
    free(bits);
    return 0;
}
