/*
 * parparaw.h -- C ABI of the GB300 ParPaRaw parser.
 *
 * ParPaRaw (Stehle & Jacobsen, "ParPaRaw: Massively Parallel Parsing of
 * Delimiter-Separated Raw Data") parses delimiter-separated bytes on the GPU
 * without a sequential pre-pass: every chunk is simulated from every DFA
 * state at once (Sec. 3.1), the chunks' state-transition vectors are combined
 * by an exclusive scan with the composite operator (Sec. 3.1), each chunk is
 * simulated again from its now known state to tag symbols, records and
 * column offsets are scanned (Sec. 3.2), and field bytes are gathered into
 * per-column buffers and converted to the column type (Sec. 3.3).  The
 * output follows the Apache Arrow columnar layout (Sec. 5).
 *
 * Conventions for every entry point:
 *   - Plain pointers and sizes only.  "device" pointers are CUDA device
 *     memory of the current device; "host" pointers are ordinary host memory.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default).
 *   - No exception ever crosses the ABI.  The return value reports argument,
 *     allocation and launch errors; the outcome of a parse is written, on the
 *     stream, into the caller's device-side pp_parse_result.
 *   - Every device-side wait inside the kernels is bounded: if a wait expires,
 *     the parse returns PP_E_TIMEOUT in its result instead of hanging.
 */
#ifndef PARPARAW_H
#define PARPARAW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define PP_MAX_STATES 8          /* |S| of a DFA */
#define PP_MAX_GROUPS 16         /* symbol groups, catch-all included */
#define PP_MAX_SYMBOLS 16        /* distinct byte values outside the catch-all */
#define PP_MAX_COLUMNS 64        /* columns of a schema */
#define PP_MAX_STRING_COLUMNS 16 /* STRING columns of a schema */
#define PP_NO_STATE 0xFF

typedef enum pp_status {
  PP_OK = 0,
  PP_E_ARG = -1,           /* a NULL or out-of-range argument */
  PP_E_NOMEM = -2,         /* a device or host allocation failed */
  PP_E_CUDA = -3,          /* a CUDA runtime call or launch failed */
  PP_E_INVALID_INPUT = -4, /* the input entered the DFA's invalid state */
  PP_E_UNTERMINATED = -5,  /* the input ended in a non-accepting state */
  PP_E_CAPACITY = -6,      /* an output buffer is too small; sizes reported */
  PP_E_TIMEOUT = -7,       /* a bounded device-side wait expired */
  PP_E_BAD_TABLE = -8,     /* the DFA / symbol groups / schema are malformed */
  PP_E_UNSUPPORTED = -9    /* a limit of this build was exceeded */
} pp_status;

/* Per-symbol tags: the paper's three bitmap indexes (record delimiter, field
 * delimiter, control symbol) plus "part of a field value" (Sec. 3.1). */
typedef enum pp_tag {
  PP_TAG_DATA = 0,
  PP_TAG_FIELD = 1,
  PP_TAG_RECORD = 2,
  PP_TAG_CONTROL = 3
} pp_tag;

/* Column types (Sec. 3.3 type conversion).  Numeric text longer than 64 data
 * bytes, or that does not follow the syntax below, fails to convert and
 * rejects its record.
 *   PP_STRING        bytes, int64 offsets (Arrow LargeUtf8 layout)
 *   PP_INT32         -?[0-9]+, must fit int32
 *   PP_INT64         -?[0-9]+, must fit int64
 *   PP_FLOAT64       -?[0-9]+(\.[0-9]+)?, decimal significand < 2^53 and at
 *                    most 22 fraction digits; correctly rounded
 *   PP_TIMESTAMP_S   YYYY-MM-DD hh:mm:ss or YYYY-MM-DDThh:mm:ss -> int64
 *                    seconds since 1970-01-01 UTC (proleptic Gregorian)
 *   PP_DATE_D        YYYY-MM-DD -> int32 days since 1970-01-01
 *   PP_TIMESTAMP_CLF dd/Mon/yyyy:hh:mm:ss +hhmm (Common Log Format) -> int64
 *                    seconds, UTC
 *   PP_SKIP          a column that is not selected (Sec. 4.3, selecting
 *                    columns): its fields count towards the record's fields
 *                    but are neither converted nor stored; its pp_column needs
 *                    no buffers (values, offsets and validity may be NULL) */
typedef enum pp_type {
  PP_STRING = 0,
  PP_INT32 = 1,
  PP_INT64 = 2,
  PP_FLOAT64 = 3,
  PP_TIMESTAMP_S = 4,
  PP_DATE_D = 5,
  PP_TIMESTAMP_CLF = 6,
  PP_SKIP = 7
} pp_type;

/* DFA of the format (Sec. 3.1; Sec. 4.5, Table 1: one row of transitions per
 * symbol group).  All pointers are host memory, read during create only.
 *   transitions[g * num_states + s]  next state after a symbol of group g
 *                                    read in state s
 *   emit[g * num_states + s]         pp_tag of that symbol (Mealy output)
 *   invalid_state                    absorbing error state, or PP_NO_STATE;
 *                                    entering it is reported (Sec. 4.3)
 *   accept_mask                      bit s set: input may end in state s */
typedef struct pp_dfa {
  uint32_t num_states; /* 1..PP_MAX_STATES */
  uint32_t num_groups; /* 1..PP_MAX_GROUPS */
  const uint8_t* transitions;
  const uint8_t* emit;
  uint8_t start_state;
  uint8_t invalid_state;
  uint32_t accept_mask;
} pp_dfa;

/* Symbol groups (Sec. 4.5): symbols with identical transitions share a group;
 * every byte value not listed maps to `catch_all`.  Host memory. */
typedef struct pp_symbol_groups {
  uint32_t num_symbols;   /* 0..PP_MAX_SYMBOLS */
  const uint8_t* symbols; /* distinct byte values */
  const uint8_t* groups;  /* group of each symbol */
  uint8_t catch_all;
} pp_symbol_groups;

/* Schema: one pp_type per column, host memory. */
typedef struct pp_schema {
  uint32_t num_columns; /* 1..PP_MAX_COLUMNS */
  const uint32_t* types;
} pp_schema;

/* One output column, all device memory owned by the caller.
 *   values    STRING: uint8_t[values_cap]; INT32/DATE_D: int32_t[rows_cap];
 *             INT64/TIMESTAMP_*: int64_t[rows_cap]; FLOAT64: double[rows_cap]
 *   offsets   STRING only: int64_t[rows_cap + 1]; NULL otherwise
 *   validity  Arrow bitmap, LSB first, (rows_cap + 7) / 8 bytes
 * Null slots: a numeric slot holds the value of its field text when that text
 * converts and 0 otherwise; a string slot spans the bytes of its field if the
 * field was present, also in a rejected row. */
typedef struct pp_column {
  void* values;
  int64_t* offsets;
  uint8_t* validity;
  uint64_t values_cap; /* STRING: bytes available in values; else ignored */
} pp_column;

/* Outcome of one parse, written by the device at the end of the parse.
 *   status               PP_OK or one of PP_E_INVALID_INPUT,
 *                        PP_E_UNTERMINATED, PP_E_CAPACITY, PP_E_TIMEOUT
 *                        (precedence: TIMEOUT, CAPACITY, INVALID, UNTERMINATED)
 *   rows                 records emitted (rows needed on PP_E_CAPACITY)
 *   n_rejected           records kept as all-null rows (field count differs
 *                        from the schema, or a numeric field did not convert)
 *   first_invalid_offset first byte whose transition enters the invalid
 *                        state, or -1
 *   consumed             see PP_OPT_PARTIAL_INPUT
 *   values_bytes_needed  per STRING column, data bytes the input holds for it
 *                        (the values_cap that is enough), else 0 */
typedef struct pp_parse_result {
  int32_t status;
  int32_t final_state;
  int64_t rows;
  int64_t n_rejected;
  int64_t first_invalid_offset;
  int64_t consumed;  /* PP_OPT_PARTIAL_INPUT: bytes up to and including the
                        last record delimiter; else len */
  int64_t values_bytes_needed[PP_MAX_COLUMNS];
} pp_parse_result;

/* Output descriptor (host struct holding device pointers).  On
 * PP_E_CAPACITY nothing is written beyond any capacity and the result holds
 * the sizes needed for a retry.  Rows before an invalid byte are output as
 * usual; the record in progress at the end of an invalid or unterminated
 * input is not emitted. */
typedef struct pp_columns {
  uint32_t num_columns;           /* must equal the schema's */
  uint64_t rows_cap;
  pp_column cols[PP_MAX_COLUMNS];
  uint8_t* row_valid;             /* device bitmap, (rows_cap + 7) / 8 bytes */
  pp_parse_result* result;        /* device memory */
} pp_columns;

typedef struct pp_parser pp_parser;

/* Tuning options (parparaw_set_option). */
typedef enum pp_option {
  PP_OPT_TILE_CONFIG = 1,   /* tile shape, threads x bytes per thread:
                               0 = default (10); 1 = 32x16 (test); 2 = 64x48;
                               3 = 256x112 (2 blocks/SM); 4 = 128x208;
                               5 = 128x112; 6 = 128x112 (6 blocks/SM);
                               7 = 128x48; 8 = 256x80; 9 = 256x96;
                               10 = 448x64; 11 = 512x48;
                               12 = 256x112 (3 blocks/SM); 13 = 384x128;
                               14 = 448x128 */
  PP_OPT_TIMEOUT_MS = 2,    /* bound of every device-side wait (default 2000) */
  PP_OPT_GRID_LIMIT = 3,    /* 0 = one block per tile; n = at most n resident
                               blocks looping over tiles (persistent) */
  PP_OPT_PARTIAL_INPUT = 4, /* 1 = the input is one partition of a longer
                               stream (Sec. 4.4): bytes after the last record
                               delimiter are an incomplete record, not emitted
                               and not an error; result.consumed reports where
                               they start.  0 (default) = the input is whole. */
  PP_OPT_FIRST_ITEM = 5,    /* testing only: the work queue starts at this tile
                               (default 0).  The tiles before it never run, so
                               later tiles' bounded look-back waits expire and
                               the parse reports PP_E_TIMEOUT; the context stays
                               usable.  Outputs of such a parse are undefined. */
  PP_OPT_SKIP_RECORDS = 6,  /* skipping records (Sec. 4.3): the first n records
                               (0 <= n < 2^32, default 0), e.g. a header, are
                               recognised and validated but leave no row, no
                               string bytes, no conversion and no reject; row 0
                               is record n.  result.rows counts the rows left.
                               parparaw_infer skips them too. */
  PP_OPT_UTF16LE = 7        /* variable-length symbols (Sec. 4.2): 1 = the input
                               is UTF-16LE code units.  Symbol bytes b of the
                               symbol groups stand for code points U+00bb; every
                               other code unit, surrogates included, is in the
                               catch-all group, and a surrogate pair reads like
                               one catch-all symbol.  A symbol's tag covers all
                               of its bytes, string values keep their UTF-16LE
                               bytes, and numeric text converts when every code
                               point is ASCII.  Needs an input address and
                               length that are even (else parparaw_parse
                               returns PP_E_ARG), and a catch-all transition
                               that is idempotent with the same tag before and
                               after it (else PP_E_UNSUPPORTED here): then a
                               surrogate pair read as two code units parses as
                               one symbol.  Parses run with tile configurations
                               0 (10), 1 and 2 (others: PP_E_UNSUPPORTED);
                               parparaw_infer returns PP_E_UNSUPPORTED for such
                               parsers.  0 (default) = byte symbols. */
} pp_option;

typedef struct pp_parser_info {
  uint32_t num_states, num_groups, num_symbols, num_columns, num_string_columns;
  uint32_t catch_all_idempotent; /* runs of catch-all symbols collapse */
  uint32_t tile_bytes;           /* input bytes per tile of the current config */
  uint32_t threads_per_block;
} pp_parser_info;

/* Validates and copies the tables (Sec. 3.1 DFA, Sec. 4.5 symbol groups,
 * schema).  Returns PP_E_BAD_TABLE when an entry is out of range, the invalid
 * state is not absorbing, a symbol is listed twice or maps to the catch-all
 * group, or the schema has an unknown type; PP_E_UNSUPPORTED when a limit of
 * this header is exceeded.  Allocates no device memory.  The parser is
 * immutable after its options are set and may be shared across host threads
 * and streams.  *out is owned by the caller and released with
 * parparaw_destroy. */
pp_status parparaw_create(const pp_dfa* dfa, const pp_symbol_groups* groups,
                          const pp_schema* schema, pp_parser** out);

void parparaw_destroy(pp_parser* parser);

pp_status parparaw_set_option(pp_parser* parser, pp_option option, int64_t value);

pp_status parparaw_get_info(const pp_parser* parser, pp_parser_info* info);

/* Parses `len` bytes at device address `input` into `out` (Sec. 3, whole
 * pipeline), asynchronously on `stream`.  `input` and the buffers of `out`
 * are caller-owned device memory and must stay valid until the stream has
 * passed the parse; `out` itself (a host struct) is read before the call
 * returns.  The library allocates its own scratch (tile status words, fail
 * bitmaps) stream-ordered on `stream` and releases it the same way.  Returns
 * PP_E_ARG / PP_E_NOMEM / PP_E_CUDA for errors detected on the host; the parse
 * outcome is in out->result once the stream reaches it. */
pp_status parparaw_parse(const pp_parser* parser, const uint8_t* input, uint64_t len,
                         const pp_columns* out, void* stream);

/* One item of a batch: its own parser (DFA, symbol groups, schema), input
 * (device) and output descriptor (host struct holding device pointers). */
typedef struct pp_batch_item {
  const pp_parser* parser;
  const uint8_t* input;
  uint64_t len;
  const pp_columns* out;
} pp_batch_item;

/* Parses `n` independent inputs, possibly with different parsers, in one
 * persistent launch whose blocks take (input, tile) work items from a device
 * queue; each input keeps its own look-back chains.  Every item's result is
 * identical to its plain parparaw_parse.  `items` is host memory read before
 * the call returns.  The tile configuration of the batch is that of the first
 * item's parser. */
pp_status parparaw_parse_batch(const pp_batch_item* items, uint64_t n, void* stream);

/* A prepared batch: the items' descriptors (the device-side work queue of
 * (input, tile) items, tables, output columns) and their scratch, uploaded
 * once to device memory so that each parparaw_batch_launch is kernel
 * launches only.  The items' inputs and outputs must stay valid while the
 * batch is launched; their contents may change between launches. */
typedef struct pp_batch pp_batch;

/* Validates the items as parparaw_parse_batch does, allocates the batch's
 * device memory (cudaMalloc) and uploads its descriptors (synchronous copy).
 * `items` is host memory read before the call returns.  *out is owned by the
 * caller and released with parparaw_batch_destroy. */
pp_status parparaw_batch_create(const pp_batch_item* items, uint64_t n, pp_batch** out);

/* Enqueues one parse of every item of the batch on `stream` (init kernel,
 * one persistent tile kernel over all items' tiles, finalize kernel).  Launches
 * of one batch must not overlap on the device: they share its scratch. */
pp_status parparaw_batch_launch(pp_batch* batch, void* stream);

/* Frees the batch (cudaFree: call it once its launches have completed). */
void parparaw_batch_destroy(pp_batch* batch);

/* End-to-end streaming from host memory (Sec. 4.4, "End-to-End Streaming"):
 * the input lives in host memory and is parsed in partitions while the next
 * partition is copied in and the previous one's columns are copied out.
 * A streamer owns two device input buffers (each a carry-over region in
 * front of a partition), two sets of device output columns, a pinned result
 * block and three CUDA streams (copy in, parse, copy out).  Each partition
 * but the last is parsed as a partial input (PP_OPT_PARTIAL_INPUT): its bytes
 * after the last record delimiter are an incomplete record, which the device
 * reports as `consumed`; they are copied on the device into the carry-over
 * region of the other buffer and parsed again at the start of the next
 * partition, which restarts in the DFA's start state (this holds for formats
 * whose record delimiter leads back to the start state).  The host waits for
 * each partition's result only to size its copy-out and the carry-over; the
 * copies of the neighbouring partitions run meanwhile. */
typedef struct pp_streamer pp_streamer;

/* Creates a streamer for `parser` (its DFA, schema and options are copied;
 * PP_OPT_SKIP_RECORDS applies to the first partition).  partition_bytes: input
 * bytes copied in per partition (> 0); carry_bytes: the longest incomplete
 * record carried over (0 = partition_bytes).  Allocates the device buffers
 * (cudaMalloc; output columns sized for one record per 16 input bytes, grown
 * on demand), pinned host memory for the results, three streams and events
 * on the current device.  *out is released with parparaw_stream_destroy. */
pp_status parparaw_stream_create(const pp_parser* parser, uint64_t partition_bytes, uint64_t carry_bytes,
                                 pp_streamer** out);

/* The columns of one partition, in the caller's host arena.  cols[c] holds
 * host pointers (NULL for PP_SKIP columns): STRING values (values_cap =
 * bytes) and int64 offsets [rows + 1] starting at 0; numeric values [rows];
 * validity bitmaps (rows + 7) / 8 bytes, LSB first.  The partition's rows are
 * rows [row0, row0 + rows) of the whole input's parse. */
typedef struct pp_host_partition {
  int64_t rows;
  int64_t row0;
  uint64_t input_offset; /* first input byte of the partition (its carry-over included) */
  uint64_t input_bytes;  /* bytes parsed for it */
  pp_column cols[PP_MAX_COLUMNS];
  uint8_t* row_valid;
  /* device time (CUDA events on the streamer's streams, milliseconds) of the
   * partition's copy in, its parse (the launches and the result read-back)
   * and the copy out of its columns; each excludes the waits before it */
  float h2d_ms, parse_ms, d2h_ms;
} pp_host_partition;

/* Outcome of a streamed parse.
 *   status               PP_OK, or the status of the first partition that
 *                        failed (PP_E_INVALID_INPUT, PP_E_UNTERMINATED,
 *                        PP_E_TIMEOUT) -- the partitions before it, and that
 *                        partition's rows before the failure, are output; or
 *                        PP_E_CAPACITY when the arena is too small, or
 *                        PP_E_UNSUPPORTED when a record is longer than the
 *                        carry-over region
 *   num_partitions       partitions written to parts
 *   rows, n_rejected     over the partitions written
 *   first_invalid_offset in the whole input, or -1
 *   arena_bytes          arena bytes used; on PP_E_CAPACITY, the bytes that
 *                        the partitions so far plus the one that did not fit
 *                        need */
typedef struct pp_stream_result {
  int32_t status;
  uint32_t num_partitions;
  int64_t rows;
  int64_t n_rejected;
  int64_t first_invalid_offset;
  uint64_t arena_bytes;
} pp_stream_result;

/* Parses `len` bytes of host memory at `input` (pinned memory lets the
 * copies run at full speed; pageable memory works but each copy then
 * blocks) into columns carved from the host arena [arena, arena +
 * arena_bytes) (64-byte aligned pieces; pinned for speed).  `parts` (host,
 * max_parts entries, at least ceil(len / partition_bytes)) receives one entry
 * per partition.  Synchronous: returns once every partition's columns are in
 * the arena and the streamer's streams are idle.  Calls on one streamer must
 * not overlap.  Returns PP_E_ARG for bad arguments (too few parts entries
 * included), PP_E_NOMEM / PP_E_CUDA for allocation and CUDA errors; the
 * parse outcome is in *result. */
pp_status parparaw_stream_parse(pp_streamer* streamer, const uint8_t* input, uint64_t len, uint8_t* arena,
                                uint64_t arena_bytes, pp_host_partition* parts, uint64_t max_parts,
                                pp_stream_result* result);

void parparaw_stream_destroy(pp_streamer* streamer);

/* Size of the fixed device scratch behind parparaw_parse_noalloc. */
#define PP_NOALLOC_SCRATCH_BYTES (32u << 20)

/* parparaw_parse without any allocation (the paper has no counterpart; it is
 * an interface convenience).  Some callers cannot allocate device memory on
 * the call path: services that reserve all device memory up front and forbid
 * the CUDA allocator afterwards, callers that account every byte through
 * their own allocator, or latency-bound paths where an allocation may stall
 * other work on the device.  This entry point takes its scratch (tile status
 * words, reject / null bitmaps, counters) from one fixed array of
 * PP_NOALLOC_SCRATCH_BYTES in device memory that the library defines; every
 * GPU that loads the library holds that array until the process exits.  It
 * calls no cudaMalloc, cudaFree or other allocating routine.
 *   - Arguments, output layout and results are those of parparaw_parse.
 *   - Returns PP_E_UNSUPPORTED, before launching anything, when the scratch
 *     this parse needs (it grows with len / tile size, with rows_cap and with
 *     the number of numeric columns) exceeds PP_NOALLOC_SCRATCH_BYTES.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.  The address is kept for the life of the
 *     process: after cudaDeviceReset on a device the array moves, so this
 *     entry point must not be called on that device again.
 *   - Every call on a device shares the one array and it keeps the previous
 *     call's contents; each call clears what must start at zero itself.
 *     Calls whose work overlaps on the GPU (other streams, other threads)
 *     race on the array: order them, e.g. on one stream. */
pp_status parparaw_parse_noalloc(const pp_parser* parser, const uint8_t* input, uint64_t len,
                                 const pp_columns* out, void* stream);

/* Column-count and numeric type inference (Sec. 4.3, "Capabilities"): parses
 * the input with the parser's DFA and symbol groups (its schema is ignored)
 * and reports the fewest and the most fields of a record, and for every field
 * position c < PP_MAX_COLUMNS the type that holds each of its non-empty
 * fields: the widest, in the chain PP_INT32 < PP_INT64 < PP_FLOAT64 <
 * PP_STRING, of the fields' narrowest types (a field's narrowest type is the
 * first of int32, int64, float64 whose conversion accepts its text, else
 * string).  Records are found exactly as by parparaw_parse.
 *   - result: device memory, written on the stream.  status as in
 *     pp_parse_result (never PP_E_CAPACITY); records = records found;
 *     min/max_fields saturate at PP_INFER_MAX_FIELDS and are 0 without
 *     records; type[c] = PP_TYPE_NONE where position c holds no non-empty
 *     field.
 *   - Runs the default tile shape whatever PP_OPT_TILE_CONFIG says.
 *   - Returns PP_E_ARG for NULL arguments, PP_E_NOMEM / PP_E_CUDA on
 *     allocation or launch failure. */
#define PP_INFER_MAX_FIELDS 256
#define PP_TYPE_NONE 0xFF
typedef struct pp_inference {
  int32_t status;
  uint32_t min_fields, max_fields;
  uint32_t pad;
  int64_t records;
  int64_t first_invalid_offset;
  uint8_t type[PP_MAX_COLUMNS];
} pp_inference;

pp_status parparaw_infer(const pp_parser* parser, const uint8_t* input, uint64_t len,
                         pp_inference* result, void* stream);

/* Skipping rows (Sec. 4.3): the pruning pass that runs before a parse.  A
 * row is a physical line: its bytes up to and including the next
 * `terminator` byte (the last row may lack it), whatever the quoting; rows
 * count from 0.  Rows differ from records (a quoted field may span lines), so
 * rows are pruned from the raw bytes, before the DFA sees them.
 *   input[0..len)      device memory, read only.
 *   rows[0..nrows)     device memory: the rows to drop, strictly increasing;
 *                      with any other list the output is unspecified (every
 *                      access still stays in bounds).  Rows past the end are
 *                      ignored.
 *   output             device memory, capacity >= len, not overlapping input:
 *                      the bytes of every other row, in order.
 *   output_len         device memory (one uint64_t): the bytes written.
 *   scratch            device memory of scratch_bytes >=
 *                      parparaw_skip_rows_scratch_bytes(len), 16-byte aligned,
 *                      owned by the caller and not used by anything else
 *                      until the stream has passed this call.
 * Asynchronous on `stream` (a cudaStream_t, NULL = default stream); a parse
 * of output[0..*output_len) follows on the same stream once the caller has
 * read *output_len.  Returns PP_E_ARG for NULL pointers with len > 0 or a
 * scratch that is too small or misaligned, PP_E_CUDA if a launch fails. */
uint64_t parparaw_skip_rows_scratch_bytes(uint64_t len);
pp_status parparaw_skip_rows(const uint8_t* input, uint64_t len, const uint64_t* rows, uint64_t nrows,
                             uint8_t terminator, uint8_t* output, uint64_t* output_len, void* scratch,
                             uint64_t scratch_bytes, void* stream);

/* Records the two CUDA events (cudaEvent_t passed as void*) on the stream
 * immediately before and after the main parse kernel of every later parse or
 * batch made with this parser, so that a caller can time that kernel alone.
 * Pass NULL, NULL to stop. */
pp_status parparaw_set_kernel_events(pp_parser* parser, void* start_event, void* stop_event);

/* Static text for a pp_status value; never NULL. */
const char* parparaw_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* PARPARAW_H */
