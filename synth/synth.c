/*
 * synth.c -- seeded synthetic delimiter-separated inputs.
 *
 * The paper evaluates on two public datasets (yelp reviews, NYC taxi trips,
 * Sec. 5) that are not available here.  These generators write seeded
 * synthetic stand-ins with the published shape statistics (column counts,
 * types, mean record sizes, quoting) and, for small cases, the logical
 * content of every field ("truth") so tests can check a parse against what
 * was written.  They only format values; they contain no parsing logic.
 *
 * Determinism: record i of a workload depends only on (seed, i), drawn from a
 * SplitMix64 stream (Steele, Lea & Flood, OOPSLA 2014).  Records are produced
 * in fixed blocks by a thread pool and concatenated in order, so the output
 * does not depend on the number of threads.
 */
#define _GNU_SOURCE
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

enum { W_MIXED = 1, W_TRIP = 2, W_REVIEW = 3, W_LOG = 4 };

/* ------------------------------------------------------------- SplitMix64 */
typedef struct { uint64_t s; } rng_t;

static inline uint64_t sm64(rng_t* r) {
  uint64_t z = (r->s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}
static inline rng_t rng_for(uint64_t seed, uint64_t record) {
  rng_t r = {seed ^ 0x5851F42D4C957F2Dull};
  r.s += record * 0xD1B54A32D192ED03ull;
  (void)sm64(&r);
  return r;
}
static inline uint64_t below(rng_t* r, uint64_t n) { return n ? sm64(r) % n : 0; }
static inline double unif(rng_t* r) { return (double)(sm64(r) >> 11) * (1.0 / 9007199254740992.0); }
static inline int chance(rng_t* r, double p) { return unif(r) < p; }
/* approximately normal: Irwin-Hall sum of 12 uniforms */
static double gauss(rng_t* r) {
  double s = 0;
  for (int i = 0; i < 12; ++i) s += unif(r);
  return s - 6.0;
}
/* log-normal with the given mean: mu = ln(mean) - sigma^2 / 2 */
static double lognormal(rng_t* r, double mean, double sigma) {
  return exp(log(mean) - 0.5 * sigma * sigma + sigma * gauss(r));
}
/* failures before the first success, success probability p */
static uint64_t geometric(rng_t* r, double p) {
  uint64_t k = 0;
  while (!chance(r, p) && k < 1000) ++k;
  return k;
}

/* ----------------------------------------------------------------- sinks */
typedef struct {
  uint8_t* p;
  size_t n, cap;
} sink_t;

static void sink_reserve(sink_t* s, size_t add) {
  if (s->n + add <= s->cap) return;
  size_t c = s->cap ? s->cap : 4096;
  while (c < s->n + add) c *= 2;
  s->p = (uint8_t*)realloc(s->p, c);
  s->cap = c;
}
static inline void put(sink_t* s, const void* b, size_t n) {
  if (!s) return;
  sink_reserve(s, n);
  memcpy(s->p + s->n, b, n);
  s->n += n;
}
static inline void putc_(sink_t* s, uint8_t c) {
  if (!s) return;
  sink_reserve(s, 1);
  s->p[s->n++] = c;
}
static inline void puts_(sink_t* s, const char* z) { put(s, z, strlen(z)); }

/* A record writer: raw bytes go to `raw`, the logical field values to
 * `truth` as 0x1F-separated fields, 0x1E-terminated records. */
typedef struct {
  sink_t* raw;
  sink_t* truth;
  int nfield;
} rec_t;

static void field_begin(rec_t* w, char sep) {
  if (w->nfield > 0) {
    putc_(w->raw, (uint8_t)sep);
    putc_(w->truth, 0x1F);
  }
  w->nfield++;
}
/* unquoted field whose raw text equals its value */
static void field_plain(rec_t* w, char sep, const char* v, size_t n) {
  field_begin(w, sep);
  put(w->raw, v, n);
  put(w->truth, v, n);
}
/* RFC-4180 quoted field: '"' inside the value is doubled */
static void field_quoted(rec_t* w, char sep, const char* v, size_t n) {
  field_begin(w, sep);
  putc_(w->raw, '"');
  for (size_t i = 0; i < n; ++i) {
    if (v[i] == '"') putc_(w->raw, '"');
    putc_(w->raw, (uint8_t)v[i]);
  }
  putc_(w->raw, '"');
  put(w->truth, v, n);
}
/* field enclosed by open/close symbols whose content is the value */
static void field_enclosed(rec_t* w, char sep, char open, const char* v, size_t n, char close) {
  field_begin(w, sep);
  putc_(w->raw, (uint8_t)open);
  put(w->raw, v, n);
  putc_(w->raw, (uint8_t)close);
  put(w->truth, v, n);
}
static void record_end(rec_t* w, const char* eol) {
  puts_(w->raw, eol);
  putc_(w->truth, 0x1E);
  w->nfield = 0;
}

/* ------------------------------------------------------- value formatting */
static int fmt_i64(char* b, int64_t v) { return sprintf(b, "%lld", (long long)v); }

static int fmt_ts(char* b, int64_t t, char sep) {
  time_t tt = (time_t)t;
  struct tm tm;
  gmtime_r(&tt, &tm);
  return sprintf(b, "%04d-%02d-%02d%c%02d:%02d:%02d", tm.tm_year + 1900, tm.tm_mon + 1,
                 tm.tm_mday, sep, tm.tm_hour, tm.tm_min, tm.tm_sec);
}
static int fmt_date(char* b, int64_t t) {
  time_t tt = (time_t)t;
  struct tm tm;
  gmtime_r(&tt, &tm);
  return sprintf(b, "%04d-%02d-%02d", tm.tm_year + 1900, tm.tm_mon + 1, tm.tm_mday);
}
static int fmt_clf(char* b, int64_t t) {
  static const char* mon[12] = {"Jan", "Feb", "Mar", "Apr", "May", "Jun",
                                "Jul", "Aug", "Sep", "Oct", "Nov", "Dec"};
  time_t tt = (time_t)t;
  struct tm tm;
  gmtime_r(&tt, &tm);
  return sprintf(b, "%02d/%s/%04d:%02d:%02d:%02d +0000", tm.tm_mday, mon[tm.tm_mon],
                 tm.tm_year + 1900, tm.tm_hour, tm.tm_min, tm.tm_sec);
}
/* decimal with `frac` fraction digits from an integer significand */
static int fmt_fixed(char* b, int neg, uint64_t m, int frac) {
  char digits[32];
  int n = sprintf(digits, "%llu", (unsigned long long)m);
  int k = 0;
  if (neg) b[k++] = '-';
  if (frac == 0) {
    memcpy(b + k, digits, (size_t)n);
    return k + n;
  }
  int ip = n - frac;
  if (ip <= 0) {
    b[k++] = '0';
    b[k++] = '.';
    for (int i = 0; i < -ip; ++i) b[k++] = '0';
    memcpy(b + k, digits, (size_t)n);
    return k + n;
  }
  memcpy(b + k, digits, (size_t)ip);
  k += ip;
  b[k++] = '.';
  memcpy(b + k, digits + ip, (size_t)frac);
  return k + frac;
}

static const char ALNUM[] = "abcdefghijklmnopqrstuvwxyzABCDEFGHIJKLMNOPQRSTUVWXYZ0123456789";
static const char IDCH[] = "ABCDEFGHIJKLMNOPQRSTUVWXYZabcdefghijklmnopqrstuvwxyz0123456789-_";

/* short string for the mixed workload; quoted 30 % of the time, and quoted
 * strings contain ',' (20 %), '\n' (5 %) or '"' (10 %) */
static void mixed_string(rec_t* w, rng_t* r) {
  char v[48];
  int n = (int)below(r, 11);
  for (int i = 0; i < n; ++i) v[i] = (i > 0 && i + 1 < n && chance(r, 0.12)) ? ' ' : ALNUM[below(r, 62)];
  if (!chance(r, 0.30)) {
    field_plain(w, ',', v, (size_t)n);
    return;
  }
  if (chance(r, 0.20)) { int p = (int)below(r, (uint64_t)n + 1); memmove(v + p + 1, v + p, (size_t)(n - p)); v[p] = ','; ++n; }
  if (chance(r, 0.05)) { int p = (int)below(r, (uint64_t)n + 1); memmove(v + p + 1, v + p, (size_t)(n - p)); v[p] = '\n'; ++n; }
  if (chance(r, 0.10)) { int p = (int)below(r, (uint64_t)n + 1); memmove(v + p + 1, v + p, (size_t)(n - p)); v[p] = '"'; ++n; }
  field_quoted(w, ',', v, (size_t)n);
}

/* config-1 style: int32, string, int64, float64, ts, string, ts, string */
static void gen_mixed(rec_t* w, rng_t* r) {
  char b[64];
  int n;
  n = fmt_i64(b, (int64_t)(int32_t)(uint32_t)sm64(r));
  field_plain(w, ',', b, (size_t)n);
  mixed_string(w, r);
  {
    int digits = 1 + (int)below(r, 18);
    uint64_t lim = 1;
    for (int i = 0; i < digits; ++i) lim *= 10;
    int64_t v = (int64_t)below(r, lim);
    n = fmt_i64(b, chance(r, 0.5) ? -v : v);
    field_plain(w, ',', b, (size_t)n);
  }
  {
    int frac = (int)below(r, 7);
    int sig = 1 + (int)below(r, (uint64_t)(15 - frac));
    uint64_t lim = 1;
    for (int i = 0; i < sig + frac && i < 15; ++i) lim *= 10;
    n = fmt_fixed(b, chance(r, 0.5), below(r, lim), frac);
    field_plain(w, ',', b, (size_t)n);
  }
  n = fmt_ts(b, (int64_t)below(r, 2147483648ull), 'T');
  field_plain(w, ',', b, (size_t)n);
  mixed_string(w, r);
  n = fmt_ts(b, (int64_t)below(r, 2147483648ull), 'T');
  field_plain(w, ',', b, (size_t)n);
  mixed_string(w, r);
  record_end(w, "\n");
}

/* config-2 style trip record, CRLF, no quoting, 18 columns:
 * int32, ts, ts, int32, f64, int32, flag, int32, str, str, f64 x7, str */
static void gen_trip(rec_t* w, rng_t* r) {
  char b[64];
  int n;
  int64_t t0 = 1514764800 + (int64_t)below(r, 365 * 86400);
  n = fmt_i64(b, 1 + (int64_t)below(r, 300)); field_plain(w, ',', b, (size_t)n);
  n = fmt_ts(b, t0, ' '); field_plain(w, ',', b, (size_t)n);
  n = fmt_ts(b, t0 + 60 + (int64_t)below(r, 3600), ' '); field_plain(w, ',', b, (size_t)n);
  n = fmt_i64(b, 1 + (int64_t)below(r, 300)); field_plain(w, ',', b, (size_t)n);
  n = fmt_fixed(b, 0, (uint64_t)llround(lognormal(r, 15.0, 0.5) * 100.0), 2); field_plain(w, ',', b, (size_t)n);
  n = fmt_i64(b, 1 + (int64_t)below(r, 300)); field_plain(w, ',', b, (size_t)n);
  field_plain(w, ',', chance(r, 0.9) ? "N" : "Y", 1);
  n = fmt_i64(b, 1 + (int64_t)below(r, 300)); field_plain(w, ',', b, (size_t)n);
  for (int k = 0; k < 2; ++k) {
    int len = 1 + (int)below(r, 3);
    for (int i = 0; i < len; ++i) b[i] = (char)('A' + below(r, 26));
    field_plain(w, ',', b, (size_t)len);
  }
  for (int k = 0; k < 7; ++k) {
    n = fmt_fixed(b, 0, (uint64_t)llround(lognormal(r, 15.0, 0.5) * 100.0), 2);
    field_plain(w, ',', b, (size_t)n);
  }
  {
    int len = 1 + (int)below(r, 3);
    for (int i = 0; i < len; ++i) b[i] = (char)('A' + below(r, 26));
    field_plain(w, ',', b, (size_t)len);
  }
  record_end(w, "\r\n");
}

/* review text: words, sentences; 40 % contain commas, 25 % line breaks,
 * 8 % double quotes; log-normal length with mean 700 bytes */
static void review_text(sink_t* t, rng_t* r) {
  size_t target = (size_t)lognormal(r, 700.0, 1.0);
  if (target < 1) target = 1;
  int commas = chance(r, 0.40), breaks = chance(r, 0.25), quotes = chance(r, 0.08);
  int word = 0;
  while (t->n < target) {
    uint64_t x = sm64(r);
    int len = 1 + (int)(x & 7);
    x >>= 3;
    sink_reserve(t, 32);
    if (word > 0) {
      uint64_t y = sm64(r);
      if (commas && (y & 15) == 0) t->p[t->n++] = ',';
      else if ((y & 31) == 1) { t->p[t->n++] = '.'; }
      else if (breaks && (y & 63) == 2) { t->p[t->n++] = '\n'; }
      if (quotes && ((y >> 8) & 63) == 3) { t->p[t->n++] = '"'; }
      t->p[t->n++] = ' ';
    }
    for (int i = 0; i < len; ++i) {
      t->p[t->n++] = (char)('a' + (x % 26));
      x /= 26;
    }
    ++word;
  }
  t->n = target;
  /* make the requested features present in short texts too */
  if (commas) t->p[target / 2] = ',';
  if (breaks && target > 2) t->p[target / 3] = '\n';
  if (quotes && target > 3) t->p[target / 4] = '"';
}

/* config-3 style review record, LF, 9 columns:
 * id x3 (22 chars), int32 stars 1-5, int32 x3 geometric(0.3), quoted text, date */
static void gen_review(rec_t* w, rng_t* r) {
  char b[64];
  int n;
  for (int k = 0; k < 3; ++k) {
    uint64_t x = sm64(r), y = sm64(r);
    for (int i = 0; i < 22; ++i) {
      uint64_t* z = i < 11 ? &x : &y;
      b[i] = IDCH[*z & 63];
      *z >>= 6;
    }
    field_plain(w, ',', b, 22);
  }
  n = fmt_i64(b, 1 + (int64_t)below(r, 5)); field_plain(w, ',', b, (size_t)n);
  for (int k = 0; k < 3; ++k) {
    n = fmt_i64(b, (int64_t)geometric(r, 0.3));
    field_plain(w, ',', b, (size_t)n);
  }
  sink_t text = {0, 0, 0};
  review_text(&text, r);
  field_quoted(w, ',', (const char*)text.p, text.n);
  free(text.p);
  n = fmt_date(b, 1104537600 + (int64_t)below(r, 15 * 365) * 86400); field_plain(w, ',', b, (size_t)n);
  record_end(w, "\n");
}

/* web-log line (Common Log Format), 7 fields separated by ' ':
 * IPv4, '-', user, [timestamp], "request", status, bytes */
static void gen_log(rec_t* w, rng_t* r) {
  static const char* methods[3] = {"GET", "POST", "HEAD"};
  static const int statuses[4] = {200, 304, 404, 500};
  char b[256];
  int n;
  uint64_t x = sm64(r);
  n = sprintf(b, "%u.%u.%u.%u", (unsigned)(x & 255), (unsigned)((x >> 8) & 255),
              (unsigned)((x >> 16) & 255), (unsigned)((x >> 24) & 255));
  field_plain(w, ' ', b, (size_t)n);
  field_plain(w, ' ', "-", 1);
  if (chance(r, 0.3)) {
    field_plain(w, ' ', "-", 1);
  } else {
    int len = 3 + (int)below(r, 8);
    for (int i = 0; i < len; ++i) b[i] = ALNUM[below(r, 26)];
    field_plain(w, ' ', b, (size_t)len);
  }
  n = fmt_clf(b, 946684800 + (int64_t)below(r, 20ull * 365 * 86400));
  field_enclosed(w, ' ', '[', b, (size_t)n, ']');
  n = sprintf(b, "%s ", methods[below(r, 3)]);
  int segs = 1 + (int)below(r, 4);
  for (int s = 0; s < segs; ++s) {
    b[n++] = '/';
    int len = 1 + (int)below(r, 10);
    for (int i = 0; i < len; ++i) b[n++] = ALNUM[below(r, 62)];
  }
  n += sprintf(b + n, " HTTP/1.1");
  field_enclosed(w, ' ', '"', b, (size_t)n, '"');
  n = fmt_i64(b, statuses[below(r, 4)]); field_plain(w, ' ', b, (size_t)n);
  n = fmt_i64(b, (int64_t)lognormal(r, 5000.0, 1.5)); field_plain(w, ' ', b, (size_t)n);
  record_end(w, "\n");
}

static void gen_record(int workload, uint64_t seed, uint64_t row, sink_t* raw, sink_t* truth) {
  rng_t r = rng_for(seed, row);
  rec_t w = {raw, truth, 0};
  switch (workload) {
    case W_MIXED: gen_mixed(&w, &r); break;
    case W_TRIP: gen_trip(&w, &r); break;
    case W_REVIEW: gen_review(&w, &r); break;
    case W_LOG: gen_log(&w, &r); break;
    default: break;
  }
}

/* -------------------------------------------------- parallel block driver */
#define BLOCK_ROWS 1024

typedef struct {
  sink_t raw;
  uint32_t ends[BLOCK_ROWS]; /* end offset of each record inside the block */
} block_t;

typedef struct {
  int workload;
  uint64_t seed;
  block_t* blocks;
  uint64_t first_block, nblocks;
  uint64_t next; /* work counter */
  pthread_mutex_t mu;
} job_t;

static void* worker(void* arg) {
  job_t* j = (job_t*)arg;
  for (;;) {
    pthread_mutex_lock(&j->mu);
    uint64_t b = j->next++;
    pthread_mutex_unlock(&j->mu);
    if (b >= j->nblocks) break;
    block_t* bl = &j->blocks[b];
    uint64_t row0 = (j->first_block + b) * BLOCK_ROWS;
    for (int i = 0; i < BLOCK_ROWS; ++i) {
      gen_record(j->workload, j->seed, row0 + (uint64_t)i, &bl->raw, NULL);
      bl->ends[i] = (uint32_t)bl->raw.n;
    }
  }
  return NULL;
}

/* Writes the longest prefix of whole records whose length is <= target_len
 * into out (capacity cap).  Returns the length written, or -1 if cap is too
 * small; *rows_out receives the record count. */
int64_t synth_generate(int workload, uint64_t seed, uint64_t target_len, uint8_t* out,
                       uint64_t cap, int threads, uint64_t* rows_out) {
  if (threads < 1) threads = 1;
  uint64_t written = 0, rows = 0, first_block = 0;
  int done = 0;
  while (!done) {
    uint64_t nb = (uint64_t)threads * 4;
    block_t* blocks = (block_t*)calloc(nb, sizeof(block_t));
    job_t j = {workload, seed, blocks, first_block, nb, 0, PTHREAD_MUTEX_INITIALIZER};
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
    for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, worker, &j);
    for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
    free(th);
    for (uint64_t b = 0; b < nb && !done; ++b) {
      block_t* bl = &blocks[b];
      uint64_t take = bl->raw.n;
      int nrec = BLOCK_ROWS;
      if (written + take > target_len) {
        nrec = 0;
        while (nrec < BLOCK_ROWS && written + bl->ends[nrec] <= target_len) ++nrec;
        take = nrec ? bl->ends[nrec - 1] : 0;
        done = 1;
      }
      if (written + take > cap) {
        for (uint64_t k = 0; k < nb; ++k) free(blocks[k].raw.p);
        free(blocks);
        return -1;
      }
      memcpy(out + written, bl->raw.p, take);
      written += take;
      rows += (uint64_t)nrec;
    }
    for (uint64_t k = 0; k < nb; ++k) free(blocks[k].raw.p);
    free(blocks);
    first_block += nb;
  }
  if (rows_out) *rows_out = rows;
  return (int64_t)written;
}

/* Raw bytes and logical field values of records [row0, row0 + nrows).
 * Returns 0, or -1 if a capacity is too small; lengths go to raw_len and truth_len. */
int synth_records(int workload, uint64_t seed, uint64_t row0, uint64_t nrows, uint8_t* raw,
                  uint64_t raw_cap, uint64_t* raw_len, uint8_t* truth, uint64_t truth_cap,
                  uint64_t* truth_len) {
  sink_t a = {0, 0, 0}, b = {0, 0, 0};
  for (uint64_t i = 0; i < nrows; ++i) gen_record(workload, seed, row0 + i, &a, &b);
  int rc = 0;
  if (a.n > raw_cap || b.n > truth_cap) rc = -1;
  else {
    memcpy(raw, a.p, a.n);
    memcpy(truth, b.p, b.n);
  }
  *raw_len = a.n;
  *truth_len = b.n;
  free(a.p);
  free(b.p);
  return rc;
}

/* ------------------------------------------------------ batches of inputs */
typedef struct {
  const int* workloads;
  const uint64_t* seeds;
  const uint64_t* targets;
  const uint64_t* offsets; /* where input i starts in out */
  uint8_t* out;
  uint64_t* lens;
  uint64_t* rows;
  uint64_t n;
  uint64_t next;
  pthread_mutex_t mu;
} batch_job_t;

static void* batch_worker(void* arg) {
  batch_job_t* b = (batch_job_t*)arg;
  for (;;) {
    pthread_mutex_lock(&b->mu);
    uint64_t i = b->next++;
    pthread_mutex_unlock(&b->mu);
    if (i >= b->n) break;
    uint64_t rows = 0;
    int64_t len = synth_generate(b->workloads[i], b->seeds[i], b->targets[i], b->out + b->offsets[i],
                                 b->targets[i], 1, &rows);
    b->lens[i] = len < 0 ? 0 : (uint64_t)len;
    b->rows[i] = rows;
  }
  return NULL;
}

/* Generates n independent inputs in parallel: input i (workload, seed) is the
 * longest whole-record prefix of length <= targets[i], written at
 * out + offsets[i] (the caller leaves targets[i] bytes there). */
void synth_generate_batch(const int* workloads, const uint64_t* seeds, const uint64_t* targets,
                          const uint64_t* offsets, uint64_t n, uint8_t* out, uint64_t* lens,
                          uint64_t* rows, int threads) {
  if (threads < 1) threads = 1;
  batch_job_t b = {workloads, seeds, targets, offsets, out, lens, rows, n, 0, PTHREAD_MUTEX_INITIALIZER};
  pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)threads);
  for (int t = 0; t < threads; ++t) pthread_create(&th[t], NULL, batch_worker, &b);
  for (int t = 0; t < threads; ++t) pthread_join(th[t], NULL);
  free(th);
}
