/*
 * orand_oracle.c -- plain, slow, obviously-correct CPU oracle for the
 * counter-based generation hot path of OpenRAND (arXiv 2310.19925).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; every constant below is written out here
 * from the primary publication the paper cites for each generator (§3).
 *
 * Precision: integer words exactly; floating point in FP64 (normals, walks,
 * adjoint).  No blocking, fusion or reordering beyond the definitions.
 *
 * Generator definitions (the paper names the generators in §3 and cites):
 *   Philox4x32-10, Threefry4x32-20  -- Salmon, Moraes, Dror, Shaw, "Parallel
 *                                      random numbers: as easy as 1, 2, 3",
 *                                      SC'11.
 *   Squares (32-bit output)          -- Widynski, "Squares: a fast
 *                                      counter-based RNG", arXiv 2004.06278.
 *   Tyche                            -- Neves & Araujo, "Fast and small
 *                                      nonlinear pseudorandom number
 *                                      generators for computer simulation",
 *                                      PPAM 2011.
 *
 * Stream identity (§2, §3): a stream is named by a 64-bit seed and a 32-bit
 * counter; the generator's internal position (block index, word index or
 * MIX count) walks the 2^32-word period of that stream.
 *
 * Pins (see tests/test_oracle_pins.py): Philox against cuRAND's host Philox
 * generator run as a black box; Tyche's MIX against ChaCha20 from the
 * `cryptography` package; Tyche and Philox constants against their closed
 * forms; the Squares key's MurmurHash3 finaliser against MurmurHash3_x64_128
 * built from the source scikit-learn ships; maps and Box-Muller against exact
 * edge values and invariants; walks against closed forms and finite
 * differences.  Threefry4x32-20's rotation
 * table and injection order and Squares' round order have no outside
 * implementation to compare with here: parity unpinned for those round
 * functions (they are checked by invariants only).
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>
#include <string.h>

/* Generator and dtype ids used by this oracle's own C interface. */
enum { ORC_PHILOX = 0, ORC_THREEFRY = 1, ORC_SQUARES = 2, ORC_TYCHE = 3 };
enum { ORC_U32 = 0, ORC_F32_UNIFORM = 1, ORC_F64_UNIFORM = 2, ORC_F32_NORMAL = 3 };

static uint32_t rotl32(uint32_t x, unsigned r)
{
    r &= 31u;
    if (r == 0) return x;
    return (x << r) | (x >> (32u - r));
}

/* ------------------------------------------------------------------------
 * Philox4x32-10 (Salmon et al. 2011).  State: four 32-bit counter words
 * c0..c3 and two key words k0,k1.  One round: multiply c0 by 0xD2511F53 and
 * c2 by 0xCD9E8D57 as full 64-bit products; the new state is
 * (hi(c2*M1) ^ c1 ^ k0, lo(c2*M1), hi(c0*M0) ^ c3 ^ k1, lo(c0*M0)).
 * Between rounds the key is bumped by the Weyl constants 0x9E3779B9 (golden
 * ratio) and 0xBB67AE85 (sqrt(3)-1).  Ten rounds.
 * ---------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 = k0 + 0x9E3779B9u;
            k1 = k1 + 0xBB67AE85u;
        }
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* ------------------------------------------------------------------------
 * Threefry4x32-20 (Salmon et al. 2011).  Key schedule: ks0..ks3 = key,
 * ks4 = 0x1BD11BDA ^ ks0 ^ ks1 ^ ks2 ^ ks3.  Start x_j = ctr_j + ks_j.
 * Round r uses rotation pair R[r mod 8]; even rounds mix (x0,x1),(x2,x3),
 * odd rounds mix (x0,x3),(x2,x1): add, rotate the second word, xor with the
 * first.  After every fourth round (injection i = 1..5) add ks_{(i+j) mod 5}
 * to x_j and add i to x3.
 * ---------------------------------------------------------------------- */
static const unsigned THREEFRY_ROT[8][2] = {
    {10, 26}, {11, 21}, {13, 27}, {23, 5}, {6, 20}, {17, 11}, {25, 10}, {18, 20}};

void orc_threefry4x32_20(const uint32_t ctr[4], const uint32_t key[4], uint32_t out[4])
{
    uint32_t ks[5];
    ks[4] = 0x1BD11BDAu;
    for (int j = 0; j < 4; ++j) {
        ks[j] = key[j];
        ks[4] ^= key[j];
    }
    uint32_t x[4];
    for (int j = 0; j < 4; ++j) x[j] = ctr[j] + ks[j];
    for (int r = 0; r < 20; ++r) {
        const unsigned ra = THREEFRY_ROT[r % 8][0], rb = THREEFRY_ROT[r % 8][1];
        if (r % 2 == 0) {
            x[0] += x[1]; x[1] = rotl32(x[1], ra) ^ x[0];
            x[2] += x[3]; x[3] = rotl32(x[3], rb) ^ x[2];
        } else {
            x[0] += x[3]; x[3] = rotl32(x[3], ra) ^ x[0];
            x[2] += x[1]; x[1] = rotl32(x[1], rb) ^ x[2];
        }
        if (r % 4 == 3) {
            uint32_t inj = (uint32_t)((r + 1) / 4);
            for (int j = 0; j < 4; ++j) x[j] += ks[(inj + (uint32_t)j) % 5u];
            x[3] += inj;
        }
    }
    for (int j = 0; j < 4; ++j) out[j] = x[j];
}

/* ------------------------------------------------------------------------
 * Squares, 32-bit output, four rounds (Widynski 2020).  All arithmetic is
 * modulo 2^64.  x = y = ctr*key, z = y + key; three rounds of
 * x = x*x + (y or z), then swap the 32-bit halves; the output is the high
 * half of x*x + z.
 * ---------------------------------------------------------------------- */
static uint64_t swap_halves(uint64_t v) { return (v >> 32) | (v << 32); }

uint32_t orc_squares32(uint64_t ctr, uint64_t key)
{
    uint64_t x = ctr * key;
    uint64_t y = x;
    uint64_t z = y + key;
    x = x * x + y; x = swap_halves(x);
    x = x * x + z; x = swap_halves(x);
    x = x * x + y; x = swap_halves(x);
    return (uint32_t)((x * x + z) >> 32);
}

/* Squares takes one 64-bit key per stream.  The paper's library accepts
 * 32-bit seeds for Squares (§3, footnote); the reading taken here derives
 * the key from the 64-bit stream key with the published MurmurHash3 64-bit
 * finaliser (Appleby) and forces it odd: key = fmix64(key64) | 1. */
uint64_t orc_squares_key(uint64_t key64)
{
    uint64_t h = key64;
    h ^= h >> 33;
    h *= 0xFF51AFD7ED558CCDull;
    h ^= h >> 33;
    h *= 0xC4CEB9FE1A85EC53ull;
    h ^= h >> 33;
    return h | 1ull;
}

/* ------------------------------------------------------------------------
 * Tyche (Neves & Araujo 2011).  State (a, b, c, d).  MIX is the ChaCha
 * quarter-round: a+=b; d=rotl(d^a,16); c+=d; b=rotl(b^c,12); a+=b;
 * d=rotl(d^a,8); c+=d; b=rotl(b^c,7).  Initialisation: a = high 32 bits of
 * the seed, b = low 32 bits, c = floor(2^32/phi) = 2654435769,
 * d = floor(2^32/pi) = 1367130551 xor the stream index (here: the counter),
 * followed by 20 MIX.  Each output word: one MIX, then return b.
 * ---------------------------------------------------------------------- */
void orc_tyche_mix(uint32_t st[4])
{
    uint32_t a = st[0], b = st[1], c = st[2], d = st[3];
    a = a + b; d = rotl32(d ^ a, 16);
    c = c + d; b = rotl32(b ^ c, 12);
    a = a + b; d = rotl32(d ^ a, 8);
    c = c + d; b = rotl32(b ^ c, 7);
    st[0] = a; st[1] = b; st[2] = c; st[3] = d;
}

void orc_tyche_init(uint64_t key64, uint32_t counter, uint32_t st[4])
{
    st[0] = (uint32_t)(key64 >> 32);
    st[1] = (uint32_t)(key64 & 0xFFFFFFFFull);
    st[2] = 2654435769u;
    st[3] = 1367130551u ^ counter;
    for (int i = 0; i < 20; ++i) orc_tyche_mix(st);
}

/* ------------------------------------------------------------------------
 * Word stream of one (generator, key64, counter) stream: words
 * [first, first + n) of its 2^32-word period.
 *   Philox:   key = (lo32(key64), hi32(key64)); word w is lane w mod 4 of the
 *             block with counter (w div 4, counter, 0, 0).
 *   Threefry: key = (lo32, hi32, 0, 0); same counter layout as Philox.
 *   Squares:  word w = squares32((counter << 32) | w, squares_key(key64)).
 *   Tyche:    word w is the output after w+1 MIX past initialisation.
 * Returns 0, or -1 for an unknown generator / a range past 2^32 words.
 * ---------------------------------------------------------------------- */
int orc_stream_words(int gen, uint64_t key64, uint32_t counter, uint64_t first, uint64_t n,
                     uint32_t *out)
{
    if (n == 0) return 0;
    if (first > (1ull << 32) || n > (1ull << 32) - first) return -1;
    const uint32_t klo = (uint32_t)(key64 & 0xFFFFFFFFull), khi = (uint32_t)(key64 >> 32);
    if (gen == ORC_PHILOX || gen == ORC_THREEFRY) {
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t w = first + i;
            uint32_t ctr[4] = {(uint32_t)(w / 4), counter, 0u, 0u};
            uint32_t blk[4];
            if (gen == ORC_PHILOX) {
                uint32_t key[2] = {klo, khi};
                orc_philox4x32_10(ctr, key, blk);
            } else {
                uint32_t key[4] = {klo, khi, 0u, 0u};
                orc_threefry4x32_20(ctr, key, blk);
            }
            out[i] = blk[w % 4];
        }
        return 0;
    }
    if (gen == ORC_SQUARES) {
        uint64_t key = orc_squares_key(key64);
        for (uint64_t i = 0; i < n; ++i) {
            uint64_t w = first + i;
            out[i] = orc_squares32(((uint64_t)counter << 32) | w, key);
        }
        return 0;
    }
    if (gen == ORC_TYCHE) {
        uint32_t st[4];
        orc_tyche_init(key64, counter, st);
        for (uint64_t w = 0; w < first; ++w) orc_tyche_mix(st);
        for (uint64_t i = 0; i < n; ++i) {
            orc_tyche_mix(st);
            out[i] = st[1];
        }
        return 0;
    }
    return -1;
}

/* ------------------------------------------------------------------------
 * Word -> value maps.
 *   FP32 uniform: (w >> 8) * 2^-24, exact, in [0, 1 - 2^-24].
 *   FP64 uniform: two words, the first one high (as in the paper's
 *                 Random123 example, Fig. 3): ((hi << 32 | lo) >> 11) * 2^-53,
 *                 exact, in [0, 1).
 *   Box-Muller:   u1 = ((w0 >> 8) + 1) * 2^-24 in (0, 1],
 *                 u2 = (w1 >> 8) * 2^-24 in [0, 1);
 *                 r = sqrt(-2 ln u1); z0 = r cos(2 pi u2), z1 = r sin(2 pi u2),
 *                 the trigonometric pair taken by exact quadrant reduction.
 * ---------------------------------------------------------------------- */
double orc_f32_uniform(uint32_t w) { return ldexp((double)(w >> 8), -24); }

double orc_f64_uniform(uint32_t hi, uint32_t lo)
{
    uint64_t v = ((uint64_t)hi << 32) | (uint64_t)lo;
    return ldexp((double)(v >> 11), -53);
}

/* cos(2 pi u2) and sin(2 pi u2) for u2 in [0, 1), by the exact quadrant
 * identity: with y = 4 u2 (exact), q = nearest integer to y and
 * t = y - q in [-1/2, 1/2] (exact), 2 pi u2 = (pi/2) q + (pi/2) t, so the pair
 * is a signed swap of (cos, sin)((pi/2) t) chosen by q mod 4.  Where the
 * exact value is 0 (u2 a multiple of 1/4) this gives exactly 0, which a
 * direct cos(2*pi*u2) in FP64 does not. */
static void cos_sin_2pi(double u2, double *c, double *s)
{
    const double half_pi = 1.5707963267948966192313216916398;
    const double y = 4.0 * u2;
    const double q = floor(y + 0.5);
    const double t = y - q;
    const double ct = cos(half_pi * t), st = sin(half_pi * t);
    switch (((long)q) & 3) {
    case 0: *c = ct; *s = st; break;
    case 1: *c = -st; *s = ct; break;
    case 2: *c = -ct; *s = -st; break;
    default: *c = st; *s = -ct; break;
    }
}

void orc_box_muller(uint32_t w0, uint32_t w1, double z[2])
{
    double u1 = ldexp((double)((w0 >> 8) + 1u), -24);
    double u2 = ldexp((double)(w1 >> 8), -24);
    double r = sqrt(-2.0 * log(u1));
    double c, s;
    cos_sin_2pi(u2, &c, &s);
    z[0] = r * c;
    z[1] = r * s;
}

/* Box-Muller over arrays of word pairs: z[2i], z[2i+1] from (w0[i], w1[i]). */
void orc_box_muller_array(const uint32_t *w0, const uint32_t *w1, uint64_t n, double *z)
{
    for (uint64_t i = 0; i < n; ++i) orc_box_muller(w0[i], w1[i], z + 2 * i);
}

/* Word -> value map over an array of words, as the fills apply it: u32
 * copies, FP32 uniform per word, FP64 uniform per word pair (first high),
 * FP32 normal per word pair.  n_values values are written (as uint32 or
 * double). */
int orc_map_words(int dtype, const uint32_t *w, uint64_t n_values, void *out)
{
    for (uint64_t j = 0; j < n_values; ++j) {
        if (dtype == ORC_U32) {
            ((uint32_t *)out)[j] = w[j];
        } else if (dtype == ORC_F32_UNIFORM) {
            ((double *)out)[j] = orc_f32_uniform(w[j]);
        } else if (dtype == ORC_F64_UNIFORM) {
            ((double *)out)[j] = orc_f64_uniform(w[2 * j], w[2 * j + 1]);
        } else if (dtype == ORC_F32_NORMAL) {
            double z[2];
            orc_box_muller(w[2 * (j / 2)], w[2 * (j / 2) + 1], z);
            ((double *)out)[j] = z[j % 2];
        } else {
            return -1;
        }
    }
    return 0;
}

/* Number of generator words a stream of `dps` values of `dtype` consumes. */
static uint64_t words_for(int dtype, uint64_t dps)
{
    if (dtype == ORC_F64_UNIFORM) return 2 * dps;
    if (dtype == ORC_F32_NORMAL) return 2 * ((dps + 1) / 2);
    return dps;
}

/* ------------------------------------------------------------------------
 * Bulk fill (one stream per processing element, §3): streams
 * s = s_first .. s_first + n_streams - 1 each get key64 = seed ^ s and the
 * user counter; stream s writes values [0, dps) at out[(s - s_first)*dps + j].
 * Output element type: uint32_t for U32, double for every float dtype
 * (FP32 uniforms are exact in double; normals stay unrounded FP64).
 * Returns 0, or -1 on an unknown generator/dtype or a stream past 2^32 words.
 * ---------------------------------------------------------------------- */
int orc_fill(int gen, int dtype, uint64_t seed, uint32_t counter, uint64_t s_first,
             uint64_t n_streams, uint64_t dps, void *out, uint32_t *word_scratch)
{
    if (dtype < ORC_U32 || dtype > ORC_F32_NORMAL) return -1;
    const uint64_t nw = words_for(dtype, dps);
    for (uint64_t i = 0; i < n_streams; ++i) {
        const uint64_t key64 = seed ^ (s_first + i);
        if (orc_stream_words(gen, key64, counter, 0, nw, word_scratch) != 0) return -1;
        for (uint64_t j = 0; j < dps; ++j) {
            const uint64_t o = i * dps + j;
            if (dtype == ORC_U32) {
                ((uint32_t *)out)[o] = word_scratch[j];
            } else if (dtype == ORC_F32_UNIFORM) {
                ((double *)out)[o] = orc_f32_uniform(word_scratch[j]);
            } else if (dtype == ORC_F64_UNIFORM) {
                ((double *)out)[o] = orc_f64_uniform(word_scratch[2 * j], word_scratch[2 * j + 1]);
            } else {
                double z[2];
                orc_box_muller(word_scratch[2 * (j / 2)], word_scratch[2 * (j / 2) + 1], z);
                ((double *)out)[o] = z[j % 2];
            }
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------
 * Fused 2D Brownian walk (the paper's macro-benchmark, Fig. 1 and §5, in
 * its pure-diffusion form).  Particle p uses key64 = seed ^ p.  Counter 0
 * gives the initial position (u(w0), u(w1)) of the first Philox block;
 * step t = 1..steps uses counter t: (z0, z1) = Box-Muller(w0, w1) of block
 * (0, t, 0, 0), and x += s*z0, y += s*z1 with s = sqrt(2 D dt).  dt and D
 * are the FP32 parameters taken as exact doubles; everything is FP64.
 * ---------------------------------------------------------------------- */
void orc_walk2d(uint64_t seed, uint64_t p_first, uint64_t n, uint32_t steps, float dt, float D,
                double *x0, double *xT)
{
    const double s = sqrt(2.0 * (double)D * (double)dt);
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t key64 = seed ^ (p_first + i);
        const uint32_t key[2] = {(uint32_t)(key64 & 0xFFFFFFFFull), (uint32_t)(key64 >> 32)};
        uint32_t blk[4];
        uint32_t ctr0[4] = {0u, 0u, 0u, 0u};
        orc_philox4x32_10(ctr0, key, blk);
        double x = orc_f32_uniform(blk[0]);
        double y = orc_f32_uniform(blk[1]);
        if (x0) { x0[2 * i] = x; x0[2 * i + 1] = y; }
        for (uint32_t t = 1; t <= steps; ++t) {
            uint32_t ctr[4] = {0u, t, 0u, 0u};
            orc_philox4x32_10(ctr, key, blk);
            double z[2];
            orc_box_muller(blk[0], blk[1], z);
            x = x + s * z[0];
            y = y + s * z[1];
        }
        xT[2 * i] = x;
        xT[2 * i + 1] = y;
    }
}

/* ------------------------------------------------------------------------
 * 3D Brownian walk with constant drift.
 * x_{t+1} = x_t + mu*dt + sigma*sqrt(dt)*z_t for t = 0..steps-1, where z_t
 * are the first three Box-Muller normals of Philox block (0, t+1, 0, 0)
 * keyed by key64 = seed ^ p: (z0, z1) from words (0, 1), z2 the cosine
 * normal of words (2, 3).  x_0 = 2u - 1 from words 0..2 of block (0, 0, 0, 0)
 * unless x0_in is given.  ckpt (nullable) receives x_{jK} for
 * j = 0 .. ceil(steps/K)-1, laid out [j][i][3].
 * ---------------------------------------------------------------------- */
static void walk3d_noise(const uint32_t key[2], uint32_t t_counter, double z[3])
{
    uint32_t ctr[4] = {0u, t_counter, 0u, 0u};
    uint32_t blk[4];
    orc_philox4x32_10(ctr, key, blk);
    double za[2], zb[2];
    orc_box_muller(blk[0], blk[1], za);
    orc_box_muller(blk[2], blk[3], zb);
    z[0] = za[0]; z[1] = za[1]; z[2] = zb[0];
}

void orc_walk3d_init(uint64_t seed, uint64_t p_first, uint64_t n, double *x0)
{
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t key64 = seed ^ (p_first + i);
        const uint32_t key[2] = {(uint32_t)(key64 & 0xFFFFFFFFull), (uint32_t)(key64 >> 32)};
        uint32_t ctr0[4] = {0u, 0u, 0u, 0u}, blk[4];
        orc_philox4x32_10(ctr0, key, blk);
        for (int c = 0; c < 3; ++c) x0[3 * i + c] = 2.0 * orc_f32_uniform(blk[c]) - 1.0;
    }
}

void orc_walk3d_forward(uint64_t seed, uint64_t p_first, uint64_t n, uint32_t steps,
                        uint32_t K, float dt, const float mu[3], float sigma,
                        const double *x0_in, double *xT, double *ckpt)
{
    const double ddt = (double)dt;
    const double sq = sqrt(ddt);
    const uint64_t n_ck = (K == 0) ? 0 : ((uint64_t)steps + K - 1) / K;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t key64 = seed ^ (p_first + i);
        const uint32_t key[2] = {(uint32_t)(key64 & 0xFFFFFFFFull), (uint32_t)(key64 >> 32)};
        double x[3];
        if (x0_in) {
            for (int c = 0; c < 3; ++c) x[c] = x0_in[3 * i + c];
        } else {
            orc_walk3d_init(seed, p_first + i, 1, x);
        }
        for (uint32_t t = 0; t < steps; ++t) {
            if (ckpt && K && t % K == 0) {
                const uint64_t j = t / K;
                for (int c = 0; c < 3; ++c) ckpt[(j * n + i) * 3 + c] = x[c];
            }
            double z[3];
            walk3d_noise(key, t + 1u, z);
            for (int c = 0; c < 3; ++c)
                x[c] = x[c] + (double)mu[c] * ddt + (double)sigma * sq * z[c];
        }
        (void)n_ck;
        for (int c = 0; c < 3; ++c) xT[3 * i + c] = x[c];
    }
}

/* Loss L = (1/P) sum_p 0.5 k |x_T,p|^2 over the n given particles, with P the
 * total particle count of the problem (so subsets add up). */
double orc_walk3d_loss(const double *xT, uint64_t n, double k, double P)
{
    double acc = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        double r2 = xT[3 * i] * xT[3 * i] + xT[3 * i + 1] * xT[3 * i + 1] +
                    xT[3 * i + 2] * xT[3 * i + 2];
        acc += 0.5 * k * r2;
    }
    return acc / P;
}

/* Reverse-mode adjoint of the walk and the loss, stepped backwards in time.
 * lambda_T = dL/dx_T = k x_T / P.  Since dx_{t+1}/dx_t = I for a constant
 * drift, lambda_t = lambda_{t+1}.  Each step t contributes lambda*dt to
 * dL/dmu and lambda . sqrt(dt) z_t to dL/dsigma, with z_t regenerated from
 * its (particle, t+1) key.  dL/dx_0 = lambda_0.  dmu[3] and dsigma[1] are
 * sums over the n given particles (they add up across subsets). */
void orc_walk3d_adjoint(uint64_t seed, uint64_t p_first, uint64_t n, uint32_t steps, float dt,
                        const double *xT, double k, double P, double *dmu, double *dsigma,
                        double *dx0)
{
    const double ddt = (double)dt;
    const double sq = sqrt(ddt);
    dmu[0] = dmu[1] = dmu[2] = 0.0;
    *dsigma = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t key64 = seed ^ (p_first + i);
        const uint32_t key[2] = {(uint32_t)(key64 & 0xFFFFFFFFull), (uint32_t)(key64 >> 32)};
        double lam[3];
        for (int c = 0; c < 3; ++c) lam[c] = k * xT[3 * i + c] / P;
        double gmu[3] = {0.0, 0.0, 0.0}, gsig = 0.0;
        for (uint32_t tt = steps; tt > 0; --tt) {
            const uint32_t t = tt - 1u;
            double z[3];
            walk3d_noise(key, t + 1u, z);
            for (int c = 0; c < 3; ++c) {
                gmu[c] += lam[c] * ddt;
                gsig += lam[c] * sq * z[c];
            }
        }
        for (int c = 0; c < 3; ++c) {
            dmu[c] += gmu[c];
            if (dx0) dx0[3 * i + c] = lam[c];
        }
        *dsigma += gsig;
    }
}

/* ------------------------------------------------------------------------
 * The paper's Brownian-dynamics macro-benchmark (Fig. 1, §5): particles with
 * velocity drag and a uniform random kick per step, FP64.  Particle p has
 * key64 = seed ^ p.  Counter 0 initialises it: (x, y) = draw_double2, i.e.
 * the two FP64 uniforms of the Philox block with counter (0, 0, 0, 0) (words
 * 0-1 and 2-3, first word high, as in Fig. 3), and v = 0.  Step `iter`
 * (1..steps) then does, in this order and in FP64:
 *     vx -= gamma / mass * vx * dt        (and vy)
 *     (rx, ry) = draw_double2 of block (0, iter, 0, 0)
 *     vx += (rx * 2 - 1) * sqrt_dt        (and vy)
 *     x  += vx * dt                       (and y)
 * gamma / mass and sqrt(dt) are evaluated once.  The position update is this
 * build's reading: Fig. 1 elides it ("...").  state: [n][4] = x, y, vx, vy.
 * ---------------------------------------------------------------------- */
void orc_langevin2d(uint64_t seed, uint64_t p_first, uint64_t n, uint32_t steps, double dt, double gamma,
                    double mass, double *state)
{
    const double g_over_m = gamma / mass;
    const double sqrt_dt = sqrt(dt);
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t key64 = seed ^ (p_first + i);
        const uint32_t key[2] = {(uint32_t)(key64 & 0xFFFFFFFFull), (uint32_t)(key64 >> 32)};
        uint32_t ctr0[4] = {0u, 0u, 0u, 0u}, blk[4];
        orc_philox4x32_10(ctr0, key, blk);
        double x = orc_f64_uniform(blk[0], blk[1]);
        double y = orc_f64_uniform(blk[2], blk[3]);
        double vx = 0.0, vy = 0.0;
        for (uint32_t iter = 1; iter <= steps; ++iter) {
            vx = vx - g_over_m * vx * dt;
            vy = vy - g_over_m * vy * dt;
            uint32_t ctr[4] = {0u, iter, 0u, 0u};
            orc_philox4x32_10(ctr, key, blk);
            const double rx = orc_f64_uniform(blk[0], blk[1]);
            const double ry = orc_f64_uniform(blk[2], blk[3]);
            vx = vx + (rx * 2.0 - 1.0) * sqrt_dt;
            vy = vy + (ry * 2.0 - 1.0) * sqrt_dt;
            x = x + vx * dt;
            y = y + vy * dt;
        }
        state[4 * i] = x;
        state[4 * i + 1] = y;
        state[4 * i + 2] = vx;
        state[4 * i + 3] = vy;
    }
}

/* ------------------------------------------------------------------------
 * 3D walk with an Ornstein-Uhlenbeck (x-dependent) drift:
 *   x_{t+1} = x_t + (mu - kappa x_t) dt + sigma sqrt(dt) z_t,
 * z_t as in orc_walk3d_forward.  kappa = 0 is that walk exactly.  Forward:
 * ckpt (nullable) receives x_{jK}; xs (nullable) receives every x_t,
 * t = 0..steps, laid out [t][i][3] (for the adjoint's dL/dkappa).
 * ---------------------------------------------------------------------- */
void orc_walk3d_ou_forward(uint64_t seed, uint64_t p_first, uint64_t n, uint32_t steps, uint32_t K, float dt,
                           const float mu[3], float sigma, float kappa, const double *x0_in, double *xT,
                           double *ckpt, double *xs)
{
    const double ddt = (double)dt;
    const double sq = sqrt(ddt);
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t key64 = seed ^ (p_first + i);
        const uint32_t key[2] = {(uint32_t)(key64 & 0xFFFFFFFFull), (uint32_t)(key64 >> 32)};
        double x[3];
        if (x0_in) {
            for (int c = 0; c < 3; ++c) x[c] = x0_in[3 * i + c];
        } else {
            orc_walk3d_init(seed, p_first + i, 1, x);
        }
        for (uint32_t t = 0; t < steps; ++t) {
            if (ckpt && K && t % K == 0)
                for (int c = 0; c < 3; ++c) ckpt[((uint64_t)(t / K) * n + i) * 3 + c] = x[c];
            if (xs)
                for (int c = 0; c < 3; ++c) xs[((uint64_t)t * n + i) * 3 + c] = x[c];
            double z[3];
            walk3d_noise(key, t + 1u, z);
            for (int c = 0; c < 3; ++c)
                x[c] = x[c] + ((double)mu[c] - (double)kappa * x[c]) * ddt + (double)sigma * sq * z[c];
        }
        if (xs)
            for (int c = 0; c < 3; ++c) xs[((uint64_t)steps * n + i) * 3 + c] = x[c];
        for (int c = 0; c < 3; ++c) xT[3 * i + c] = x[c];
    }
}

/* Adjoint of the OU walk, stepped backwards with the stored positions xs
 * ([t][i][3], from orc_walk3d_ou_forward):
 *   lambda_T = k x_T / P;  for t = steps-1 .. 0, with lambda = lambda_{t+1}:
 *     dL/dmu    += lambda dt
 *     dL/dsigma += lambda . sqrt(dt) z_t
 *     dL/dkappa += lambda . (-x_t dt)
 *     lambda_t   = lambda (1 - kappa dt)        (dx_{t+1}/dx_t = (1 - kappa dt) I)
 *   dL/dx0 = lambda_0.
 * Sums over the n given particles. */
void orc_walk3d_ou_adjoint(uint64_t seed, uint64_t p_first, uint64_t n, uint32_t steps, float dt, float kappa,
                           const double *xs, double k, double P, double *dmu, double *dsigma, double *dkappa,
                           double *dx0)
{
    const double ddt = (double)dt;
    const double sq = sqrt(ddt);
    const double decay = 1.0 - (double)kappa * ddt;
    dmu[0] = dmu[1] = dmu[2] = 0.0;
    *dsigma = 0.0;
    *dkappa = 0.0;
    for (uint64_t i = 0; i < n; ++i) {
        const uint64_t key64 = seed ^ (p_first + i);
        const uint32_t key[2] = {(uint32_t)(key64 & 0xFFFFFFFFull), (uint32_t)(key64 >> 32)};
        double lam[3];
        for (int c = 0; c < 3; ++c) lam[c] = k * xs[((uint64_t)steps * n + i) * 3 + c] / P;
        for (uint32_t tt = steps; tt > 0; --tt) {
            const uint32_t t = tt - 1u;
            double z[3];
            walk3d_noise(key, t + 1u, z);
            for (int c = 0; c < 3; ++c) {
                dmu[c] += lam[c] * ddt;
                *dsigma += lam[c] * sq * z[c];
                *dkappa += lam[c] * (-xs[((uint64_t)t * n + i) * 3 + c] * ddt);
                lam[c] *= decay;
            }
        }
        if (dx0)
            for (int c = 0; c < 3; ++c) dx0[3 * i + c] = lam[c];
    }
}
