/*
 * kem_oracle.c -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * Plain CPU restatement of the pieces around HQC.PKE that the KEM needs
 * (Sec. II-A: SHAKE as the sampler's PRNG, the domain-separated functions
 * G, H, K, and the HHK transform with implicit rejection; Algorithms 1-3;
 * the batched Keccak of Sec. III-C).  Linked into the same test library as
 * hqc_oracle.c and used only by tests/, the smoke check and bench.py's CPU
 * legs.  It shares nothing with the CUDA library.
 *
 * Readings (the paper names SHAKE and G, H, K but not their inputs; these
 * are this project's choices and are listed with the others):
 *   A16 SHAKE256 is the FIPS 202 sponge: Keccak-f[1600], rate 136 bytes,
 *       suffix bits 1111 then pad10*1.  Pinned against Python's hashlib.
 *   A17 fixed-weight sampler FW(n, w; R_0..R_{w-1}) on 32-bit words:
 *       pos_i = i + floor(R_i (n - i) / 2^32); then for i = w-2 down to 0,
 *       pos_i := i when pos_i already occurs among pos_{i+1..w-1}.  This is
 *       Floyd's subset-sampling algorithm in the constant-time arrangement
 *       Sendrier describes for constant-weight words; its output is a
 *       uniform w-subset when the draws are uniform over [0, n - i).
 *   A18 words R are the little-endian 32-bit words of a SHAKE256 stream.
 *       Encryption randomness: stream SHAKE256(theta || 0x01) gives r1 (w_r
 *       words), then r2 (w_r), then e (w_e), in that order.
 *   A19 theta = G(m, salt) = first 32 bytes of SHAKE256(m || salt || 0x03);
 *       salt is 16 bytes carried with the ciphertext.
 *   A20 K(x, c) = first 32 bytes of SHAKE256(x || U || V || salt || 0x04),
 *       x the k-byte message (or sigma on rejection), U the first
 *       ceil(n/8) bytes of u with bits >= n cleared, V the n1 n2 / 8 bytes
 *       of v.
 *   A21 Decaps: m' = Decrypt(y; u, v); (u', v') = Encrypt(pk, m'; FW(G(m',
 *       salt))); accept iff u' = u on the n bits and v' = v; K(m', c) when
 *       accepted, K(sigma, c) otherwise.  Padding bits of u are ignored,
 *       as in decryption.
 *   A22 KeyGen from seeds: h = first n bits of the stream SHAKE256(seed_pk
 *       || 0x02) (little-endian 64-bit words); x then y (w words each) from
 *       the stream SHAKE256(seed_sk || 0x01) through FW.
 * Bit-compatibility with other HQC implementations is NOT claimed: the
 * domain bytes and the order of the draws are readings, "parity unpinned"
 * against anything outside this repository.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

/* ------------------------------------------------------------------ */
/* Keccak-f[1600] (FIPS 202, Sec. 3.2): state lanes A[x][y], 64 bits,   */
/* lane (x, y) holds bytes 8 (x + 5 y) .. 8 (x + 5 y) + 7 little-endian. */
/* ------------------------------------------------------------------ */
static uint64_t rotl64(uint64_t v, int r)
{
    r &= 63;
    return r ? (v << r) | (v >> (64 - r)) : v;
}

/* rc(t): output bit of the LFSR with polynomial x^8 + x^6 + x^5 + x^4 + 1
 * after t steps (FIPS 202 Algorithm 5), the register kept as bits
 * R[0..8] with R[0] first. */
static int rc_bit(int t)
{
    if (t % 255 == 0) return 1;
    int R[9] = {1, 0, 0, 0, 0, 0, 0, 0, 0};   /* R = 10000000 */
    for (int i = 1; i <= t % 255; i++) {
        for (int j = 8; j > 0; j--) R[j] = R[j - 1];   /* R = 0 || R */
        R[0] = 0;
        R[0] ^= R[8];
        R[4] ^= R[8];
        R[5] ^= R[8];
        R[6] ^= R[8];
        R[8] = 0;                                      /* R = Trunc_8(R) */
    }
    return R[0];
}

static void keccak_f1600(uint64_t A[5][5])
{
    /* rho offsets (FIPS 202 Algorithm 2): walk (x, y) from (1, 0). */
    int rho[5][5];
    memset(rho, 0, sizeof rho);
    {
        int x = 1, y = 0;
        for (int t = 0; t < 24; t++) {
            rho[x][y] = ((t + 1) * (t + 2) / 2) % 64;
            int nx = y, ny = (2 * x + 3 * y) % 5;
            x = nx;
            y = ny;
        }
    }
    for (int ir = 0; ir < 24; ir++) {
        /* theta */
        uint64_t C[5], D[5];
        for (int x = 0; x < 5; x++)
            C[x] = A[x][0] ^ A[x][1] ^ A[x][2] ^ A[x][3] ^ A[x][4];
        for (int x = 0; x < 5; x++)
            D[x] = C[(x + 4) % 5] ^ rotl64(C[(x + 1) % 5], 1);
        for (int x = 0; x < 5; x++)
            for (int y = 0; y < 5; y++) A[x][y] ^= D[x];
        /* rho */
        for (int x = 0; x < 5; x++)
            for (int y = 0; y < 5; y++) A[x][y] = rotl64(A[x][y], rho[x][y]);
        /* pi: A'[x][y] = A[(x + 3 y) mod 5][x] */
        uint64_t B[5][5];
        for (int x = 0; x < 5; x++)
            for (int y = 0; y < 5; y++) B[x][y] = A[(x + 3 * y) % 5][x];
        /* chi */
        for (int x = 0; x < 5; x++)
            for (int y = 0; y < 5; y++)
                A[x][y] = B[x][y] ^ ((~B[(x + 1) % 5][y]) & B[(x + 2) % 5][y]);
        /* iota: RC bit 2^j - 1 = rc(j + 7 ir) */
        uint64_t RC = 0;
        for (int j = 0; j <= 6; j++)
            if (rc_bit(j + 7 * ir)) RC |= (uint64_t)1 << ((1 << j) - 1);
        A[0][0] ^= RC;
    }
}

/* Exposed for the tests: one permutation on 200 bytes in place. */
void oracle_keccak_f1600(uint8_t st[200])
{
    uint64_t A[5][5];
    for (int x = 0; x < 5; x++)
        for (int y = 0; y < 5; y++) {
            uint64_t v = 0;
            for (int b = 0; b < 8; b++) v |= (uint64_t)st[8 * (x + 5 * y) + b] << (8 * b);
            A[x][y] = v;
        }
    keccak_f1600(A);
    for (int x = 0; x < 5; x++)
        for (int y = 0; y < 5; y++)
            for (int b = 0; b < 8; b++) st[8 * (x + 5 * y) + b] = (uint8_t)(A[x][y] >> (8 * b));
}

/* SHAKE256(M, 8 outlen) (FIPS 202 Sec. 6.2): the padded message
 * M || 1111 || 10*1 absorbed in 136-byte blocks, then squeezed. */
#define SHAKE256_RATE 136
void oracle_shake256(const uint8_t *msg, int64_t len, uint8_t *out, int64_t outlen)
{
    uint8_t st[200];
    memset(st, 0, sizeof st);
    const int64_t padded = (len / SHAKE256_RATE + 1) * SHAKE256_RATE;
    uint8_t *P = (uint8_t *)calloc((size_t)padded, 1);
    if (len) memcpy(P, msg, (size_t)len);
    P[len] ^= 0x1F;                 /* suffix 1111, then the first pad bit */
    P[padded - 1] ^= 0x80;          /* last pad bit */
    for (int64_t off = 0; off < padded; off += SHAKE256_RATE) {
        for (int i = 0; i < SHAKE256_RATE; i++) st[i] ^= P[off + i];
        oracle_keccak_f1600(st);
    }
    free(P);
    for (int64_t o = 0; o < outlen; o += SHAKE256_RATE) {
        int64_t take = outlen - o < SHAKE256_RATE ? outlen - o : SHAKE256_RATE;
        memcpy(out + o, st, (size_t)take);
        if (o + SHAKE256_RATE < outlen) oracle_keccak_f1600(st);
    }
}

/* ------------------------------------------------------------------ */
/* A17: fixed-weight sampler on given 32-bit draws.                     */
/* ------------------------------------------------------------------ */
void oracle_fixed_weight(int n, int w, const uint32_t *R, uint32_t *pos)
{
    for (int i = 0; i < w; i++)
        pos[i] = (uint32_t)i + (uint32_t)(((uint64_t)R[i] * (uint64_t)(n - i)) >> 32);
    for (int i = w - 2; i >= 0; i--) {
        int seen = 0;
        for (int j = i + 1; j < w; j++) seen |= pos[j] == pos[i];
        if (seen) pos[i] = (uint32_t)i;
    }
}

/* A18: w words of a SHAKE256 stream starting at word `first`. */
static void stream_words(const uint8_t *seed, int seedlen, uint8_t dom, int64_t first, int count, uint32_t *R)
{
    uint8_t *in = (uint8_t *)malloc((size_t)seedlen + 1);
    memcpy(in, seed, (size_t)seedlen);
    in[seedlen] = dom;
    const int64_t nbytes = 4 * (first + count);
    uint8_t *buf = (uint8_t *)malloc((size_t)nbytes);
    oracle_shake256(in, seedlen + 1, buf, nbytes);
    for (int i = 0; i < count; i++) {
        const uint8_t *b = buf + 4 * (first + i);
        R[i] = (uint32_t)b[0] | (uint32_t)b[1] << 8 | (uint32_t)b[2] << 16 | (uint32_t)b[3] << 24;
    }
    free(buf);
    free(in);
}

/* ------------------------------------------------------------------ */
/* KEM (A19-A22) on top of the PKE oracle of hqc_oracle.c.              */
/* ------------------------------------------------------------------ */
int oracle_params(int level, int32_t *out9);
int oracle_encrypt_batch(int level, int64_t count, const uint64_t *h, const uint64_t *s, const int32_t *key_idx,
                         const uint8_t *m, const uint32_t *r1, const uint32_t *r2, const uint32_t *e,
                         uint64_t *u_out, uint64_t *v_out, int nthreads);
int oracle_decrypt_batch(int level, int64_t count, const uint64_t *u, const uint64_t *v, const uint32_t *y,
                         uint8_t *m_out, int nthreads);
int oracle_keygen_batch(int level, int64_t nkeys, const uint64_t *h, const uint32_t *x, const uint32_t *y,
                        uint64_t *s_out, int nthreads);

typedef struct {
    int n, w, wr, we, n1, k, n2;
    int W_u, W_u_pitch, W_v, u_bytes, v_bytes;
} kparams;

static int kem_params(int level, kparams *q)
{
    int32_t o[9];
    if (oracle_params(level, o)) return -1;
    q->n = o[0]; q->w = o[1]; q->wr = o[2]; q->we = o[3]; q->n1 = o[4]; q->k = o[5]; q->n2 = o[7];
    q->W_u = (q->n + 63) / 64;
    q->W_u_pitch = q->W_u + (q->W_u & 1);
    q->W_v = q->n1 * q->n2 / 64;
    q->u_bytes = (q->n + 7) / 8;
    q->v_bytes = q->n1 * q->n2 / 8;
    return 0;
}

/* Byte i of a little-endian word array; bits >= nbits cleared. */
static uint8_t le_byte(const uint64_t *words, int i, int nbits)
{
    uint8_t b = (uint8_t)(words[i / 8] >> (8 * (i % 8)));
    const int lo = 8 * i;
    if (lo + 8 > nbits) b &= (uint8_t)((1u << (nbits > lo ? nbits - lo : 0)) - 1u);
    return b;
}

/* A19 */
void oracle_kem_theta(int k, const uint8_t *m, const uint8_t *salt, uint8_t theta[32])
{
    uint8_t in[256];
    memcpy(in, m, (size_t)k);
    memcpy(in + k, salt, 16);
    in[k + 16] = 0x03;
    oracle_shake256(in, k + 17, theta, 32);
}

/* A18: r1, r2, e from theta. */
int oracle_kem_randomness(int level, const uint8_t theta[32], uint32_t *r1, uint32_t *r2, uint32_t *e)
{
    kparams q;
    if (kem_params(level, &q)) return -1;
    const int total = 2 * q.wr + q.we;
    uint32_t *R = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)total);
    stream_words(theta, 32, 0x01, 0, total, R);
    oracle_fixed_weight(q.n, q.wr, R, r1);
    oracle_fixed_weight(q.n, q.wr, R + q.wr, r2);
    oracle_fixed_weight(q.n, q.we, R + 2 * q.wr, e);
    free(R);
    return 0;
}

/* A20 */
static void kem_K(const kparams *q, const uint8_t *x, const uint64_t *u, const uint64_t *v, const uint8_t *salt,
                  uint8_t K[32])
{
    const int len = q->k + q->u_bytes + q->v_bytes + 16 + 1;
    uint8_t *in = (uint8_t *)malloc((size_t)len);
    int o = 0;
    memcpy(in, x, (size_t)q->k);
    o += q->k;
    for (int i = 0; i < q->u_bytes; i++) in[o++] = le_byte(u, i, q->n);
    for (int i = 0; i < q->v_bytes; i++) in[o++] = le_byte(v, i, q->n1 * q->n2);
    memcpy(in + o, salt, 16);
    o += 16;
    in[o] = 0x04;
    oracle_shake256(in, len, K, 32);
    free(in);
}

/* A22: h, x, y, s from seeds.  seed_sk, seed_pk: [nkeys][32]. */
int oracle_kem_keygen(int level, int64_t nkeys, const uint8_t *seed_sk, const uint8_t *seed_pk, uint64_t *h_out,
                      uint32_t *x_out, uint32_t *y_out, uint64_t *s_out)
{
    kparams q;
    if (kem_params(level, &q)) return -1;
    for (int64_t i = 0; i < nkeys; i++) {
        uint64_t *h = h_out + i * q.W_u_pitch;
        uint8_t in[33];
        memcpy(in, seed_pk + 32 * i, 32);
        in[32] = 0x02;
        uint8_t *hb = (uint8_t *)malloc((size_t)q.W_u * 8);
        oracle_shake256(in, 33, hb, (int64_t)q.W_u * 8);
        memset(h, 0, sizeof(uint64_t) * (size_t)q.W_u_pitch);
        for (int wdx = 0; wdx < q.W_u; wdx++)
            for (int b = 0; b < 8; b++) h[wdx] |= (uint64_t)hb[8 * wdx + b] << (8 * b);
        if (q.n % 64) h[q.W_u - 1] &= ((uint64_t)1 << (q.n % 64)) - 1;
        free(hb);
        uint32_t *R = (uint32_t *)malloc(sizeof(uint32_t) * 2 * (size_t)q.w);
        stream_words(seed_sk + 32 * i, 32, 0x01, 0, 2 * q.w, R);
        oracle_fixed_weight(q.n, q.w, R, x_out + i * q.w);
        oracle_fixed_weight(q.n, q.w, R + q.w, y_out + i * q.w);
        free(R);
    }
    return oracle_keygen_batch(level, nkeys, h_out, x_out, y_out, s_out, 1);
}

/* Encaps: per item, key key_idx[i] of (h, s); m [count][k], salt
 * [count][16] -> u [count][W_u_pitch], v [count][W_v], K [count][32]. */
int oracle_kem_encaps(int level, int64_t count, const uint64_t *h, const uint64_t *s, const int32_t *key_idx,
                      const uint8_t *m, const uint8_t *salt, uint64_t *u_out, uint64_t *v_out, uint8_t *K_out)
{
    kparams q;
    if (kem_params(level, &q)) return -1;
    uint32_t *r1 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)q.wr);
    uint32_t *r2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)q.wr);
    uint32_t *e = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)q.we);
    int rc = 0;
    for (int64_t i = 0; i < count && rc == 0; i++) {
        uint8_t theta[32];
        oracle_kem_theta(q.k, m + i * q.k, salt + 16 * i, theta);
        oracle_kem_randomness(level, theta, r1, r2, e);
        uint64_t *u = u_out + i * q.W_u_pitch, *v = v_out + i * q.W_v;
        rc = oracle_encrypt_batch(level, 1, h, s, key_idx + i, m + i * q.k, r1, r2, e, u, v, 1);
        kem_K(&q, m + i * q.k, u, v, salt + 16 * i, K_out + 32 * i);
    }
    free(r1);
    free(r2);
    free(e);
    return rc;
}

/* Decaps (A21): y [nkeys][w], sigma [nkeys][k]; ok_out [count] (may be
 * NULL) receives 1 when the re-encryption matched.  Items are split over
 * nthreads threads (each item is independent). */
typedef struct {
    int level;
    int64_t first, last;
    const uint64_t *h, *s, *u_in, *v_in;
    const uint32_t *y;
    const uint8_t *sigma, *salt;
    const int32_t *key_idx;
    uint8_t *K_out;
    int32_t *ok_out;
    int rc;
} decaps_job;

static void *decaps_range(void *arg)
{
    decaps_job *J = (decaps_job *)arg;
    kparams q;
    if (kem_params(J->level, &q)) { J->rc = -1; return NULL; }
    uint32_t *r1 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)q.wr);
    uint32_t *r2 = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)q.wr);
    uint32_t *e = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)q.we);
    uint64_t *u2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)q.W_u_pitch);
    uint64_t *v2 = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)q.W_v);
    uint8_t *mp = (uint8_t *)malloc((size_t)q.k);
    int rc = 0;
    for (int64_t i = J->first; i < J->last && rc == 0; i++) {
        const int32_t key = J->key_idx[i];
        const uint64_t *u = J->u_in + i * q.W_u_pitch, *v = J->v_in + i * q.W_v;
        rc = oracle_decrypt_batch(J->level, 1, u, v, J->y + (int64_t)key * q.w, mp, 1);
        uint8_t theta[32];
        oracle_kem_theta(q.k, mp, J->salt + 16 * i, theta);
        oracle_kem_randomness(J->level, theta, r1, r2, e);
        if (rc == 0) rc = oracle_encrypt_batch(J->level, 1, J->h, J->s, &key, mp, r1, r2, e, u2, v2, 1);
        int same = 1;
        for (int b = 0; b < q.n; b++)
            same &= ((u[b / 64] >> (b % 64)) & 1) == ((u2[b / 64] >> (b % 64)) & 1);
        for (int wdx = 0; wdx < q.W_v; wdx++) same &= v[wdx] == v2[wdx];
        kem_K(&q, same ? mp : J->sigma + (int64_t)key * q.k, u, v, J->salt + 16 * i, J->K_out + 32 * i);
        if (J->ok_out) J->ok_out[i] = same;
    }
    free(r1);
    free(r2);
    free(e);
    free(u2);
    free(v2);
    free(mp);
    J->rc = rc;
    return NULL;
}

int oracle_kem_decaps(int level, int64_t count, const uint64_t *h, const uint64_t *s, const uint32_t *y,
                      const uint8_t *sigma, const int32_t *key_idx, const uint64_t *u_in, const uint64_t *v_in,
                      const uint8_t *salt, uint8_t *K_out, int32_t *ok_out, int nthreads)
{
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (count < nthreads) nthreads = count > 0 ? (int)count : 1;
    decaps_job jobs[256];
    pthread_t tid[256];
    for (int t = 0; t < nthreads; t++) {
        decaps_job *J = &jobs[t];
        J->level = level;
        J->first = count * t / nthreads;
        J->last = count * (t + 1) / nthreads;
        J->h = h; J->s = s; J->y = y; J->sigma = sigma; J->key_idx = key_idx;
        J->u_in = u_in; J->v_in = v_in; J->salt = salt; J->K_out = K_out; J->ok_out = ok_out;
        J->rc = 0;
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&tid[t], NULL, decaps_range, &jobs[t]);
    decaps_range(&jobs[0]);
    int rc = jobs[0].rc;
    for (int t = 1; t < nthreads; t++) {
        pthread_join(tid[t], NULL);
        if (jobs[t].rc) rc = jobs[t].rc;
    }
    return rc;
}
