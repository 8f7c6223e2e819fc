/*
 * synth.c -- seeded synthetic inputs for HQC.PKE key and ciphertext
 * construction.  Random numbers only: this file holds none of the scheme's
 * arithmetic (no ring product, no code), so both the CPU oracle and the
 * CUDA library can consume its output without sharing method code.
 *
 * Generators (published definitions):
 *   SplitMix64  (Steele, Lea, Flood 2014) -- seed derivation;
 *   xoshiro256** (Blackman, Vigna 2018)  -- the stream itself.
 * Uniform integers in [0, n) use plain rejection of 32-bit draws above the
 * largest multiple of n, so every value is equally likely.
 *
 * Distributions follow Algorithms 1 and 3 of the paper: h uniform over n
 * bits, supports uniform among weight-w subsets (drawn as distinct uniform
 * positions), m uniform over k bytes.
 */
#include <stdint.h>
#include <string.h>

static uint64_t splitmix64_next(uint64_t *x)
{
    uint64_t z = (*x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static inline uint64_t rotl(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

typedef struct { uint64_t s[4]; } xo_state;

static uint64_t xo_next(xo_state *st)
{
    uint64_t *s = st->s;
    uint64_t result = rotl(s[1] * 5, 7) * 9;
    uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl(s[3], 45);
    return result;
}

/* Stream for (master, level, kind, index): the four state words are
 * successive SplitMix64 outputs from a domain-separated start value. */
static void xo_seed(xo_state *st, uint64_t master, int level, int kind, uint64_t index)
{
    uint64_t x = master ^ ((uint64_t)(level & 0xff) << 56) ^ ((uint64_t)(kind & 0xff) << 48) ^ index;
    for (int i = 0; i < 4; i++) st->s[i] = splitmix64_next(&x);
}

static uint32_t uniform_below(xo_state *st, uint32_t n)
{
    uint64_t limit = (((uint64_t)1 << 32) / n) * n;
    for (;;) {
        uint64_t r = xo_next(st) >> 32;
        if (r < limit) return (uint32_t)(r % n);
    }
}

static void support(xo_state *st, uint32_t n, int w, uint32_t *out)
{
    int have = 0;
    while (have < w) {
        uint32_t p = uniform_below(st, n);
        int dup = 0;
        for (int i = 0; i < have; i++) dup |= (out[i] == p);
        if (!dup) out[have++] = p;
    }
}

enum { KIND_KEY = 1, KIND_CT = 2, KIND_SHUFFLE = 3, KIND_FREE = 4 };

/*
 * Keys: h [nkeys][wpitch] uniform n-bit (bits >= n zero), x, y [nkeys][w].
 */
void synth_keys(uint64_t master, int level, int64_t first, int64_t nkeys, int n,
                int w, int wpitch, uint64_t *h, uint32_t *x, uint32_t *y)
{
    for (int64_t i = 0; i < nkeys; i++) {
        xo_state st;
        xo_seed(&st, master, level, KIND_KEY, (uint64_t)(first + i));
        uint64_t *hr = h + i * wpitch;
        for (int j = 0; j < wpitch; j++) hr[j] = xo_next(&st);
        for (int j = 0; j < wpitch; j++) {
            int lo = j * 64;
            if (lo >= n) hr[j] = 0;
            else if (n - lo < 64) hr[j] &= (((uint64_t)1 << (n - lo)) - 1);
        }
        support(&st, (uint32_t)n, w, x + i * w);
        support(&st, (uint32_t)n, w, y + i * w);
    }
}

/*
 * Per-ciphertext randomness: m [count][k], r1, r2 [count][wr], e [count][we].
 */
void synth_ciphertexts(uint64_t master, int level, int64_t first, int64_t count,
                       int n, int k, int wr, int we, uint8_t *m, uint32_t *r1,
                       uint32_t *r2, uint32_t *e)
{
    for (int64_t i = 0; i < count; i++) {
        xo_state st;
        xo_seed(&st, master, level, KIND_CT, (uint64_t)(first + i));
        for (int j = 0; j < k; j++) m[i * k + j] = (uint8_t)(xo_next(&st) >> 56);
        support(&st, (uint32_t)n, wr, r1 + i * wr);
        support(&st, (uint32_t)n, wr, r2 + i * wr);
        support(&st, (uint32_t)n, we, e + i * we);
    }
}

/* Seeded Fisher-Yates shuffle of an int32 array. */
void synth_shuffle_i32(uint64_t master, int tag, int32_t *a, int64_t len)
{
    xo_state st;
    xo_seed(&st, master, tag, KIND_SHUFFLE, 0);
    for (int64_t i = len - 1; i > 0; i--) {
        uint64_t j = xo_next(&st) % (uint64_t)(i + 1);
        int32_t t = a[i];
        a[i] = a[j];
        a[j] = t;
    }
}

/* Raw uniform 64-bit words (garbage padding, random received words). */
void synth_words(uint64_t master, int tag, uint64_t index, uint64_t *out, int64_t len)
{
    xo_state st;
    xo_seed(&st, master, tag, KIND_FREE, index);
    for (int64_t i = 0; i < len; i++) out[i] = xo_next(&st);
}

/* Uniform integers in [0, n), e.g. random supports with repeats allowed. */
void synth_below(uint64_t master, int tag, uint64_t index, uint32_t n, uint32_t *out,
                 int64_t len)
{
    xo_state st;
    xo_seed(&st, master, tag, KIND_FREE, index ^ 0x5555555555555555ull);
    for (int64_t i = 0; i < len; i++) out[i] = uniform_below(&st, n);
}

/* Distinct positions in [0, n) (a support of weight w) for free use. */
void synth_support(uint64_t master, int tag, uint64_t index, uint32_t n, int w,
                   uint32_t *out)
{
    xo_state st;
    xo_seed(&st, master, tag, KIND_FREE, index ^ 0xAAAAAAAAAAAAAAAAull);
    support(&st, n, w, out);
}

/* First outputs of xoshiro256** seeded with explicit state, so a test can
 * compare against the generator's published reference values. */
void synth_xoshiro_raw(const uint64_t s[4], uint64_t *out, int len)
{
    xo_state st;
    memcpy(st.s, s, sizeof st.s);
    for (int i = 0; i < len; i++) out[i] = xo_next(&st);
}

void synth_splitmix_raw(uint64_t seed, uint64_t *out, int len)
{
    for (int i = 0; i < len; i++) out[i] = splitmix64_next(&seed);
}
