/*
 * anonshield.h — C ABI of the B300 pseudonymization hot path.
 *
 * The operation is the paper's problem statement (AnonShield, §2 "The
 * AnonShield Framework"): records in, pseudonymised records plus an
 * entity -> pseudonym map out, under an operator-defined key. One call runs,
 * on one GPU:
 *   byte tokenizer + pattern recognizers            (§2 stage (2))
 *   encoder-only token-classification NER           (§2 stage (2))
 *   argmax + BIO decoding + overlap rule + preserve (§2 stage (2), Appendix D)
 *   HMAC-SHA256 slug substitution                   (§2 stage (3))
 *   entity map update                               (§2 stage (4))
 *   structure-preserving output                     (§2 stage (5))
 *
 * Conventions (every entry point):
 *   - Return value: AS_OK (0) or a negative as_status; nothing is thrown.
 *     as_last_error(ctx) gives a message for the last failing call on ctx.
 *   - The caller owns every input buffer; the library reads it during the
 *     call only. The library owns every as_output and every pointer it hands
 *     out; they stay valid until the matching free call.
 *   - One as_ctx per thread (or external locking).
 *   - A ctx keeps one entity map under one key: calling with a different key
 *     while the map is non-empty is AS_ERR_STATE (same entity + same key ->
 *     same pseudonym; Fig. 1 caption).
 *   - Record index = records processed by earlier calls on this ctx +
 *     position in the call; it is the first_seen / last_seen value.
 *   - All device work runs on the ctx's stream; calls are synchronous with
 *     respect to the host (they return when results are ready).
 */
#ifndef ANONSHIELD_H
#define ANONSHIELD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t as_status;
#define AS_OK               0
#define AS_ERR_ARG         -1  /* invalid argument, size or layout          */
#define AS_ERR_OOM         -2  /* device or host allocation failed          */
#define AS_ERR_CUDA        -3  /* a CUDA call failed                        */
#define AS_ERR_TOO_LONG    -4  /* record longer than max_pos, no windows    */
#define AS_ERR_TIMEOUT     -5  /* a bounded device wait ran out             */
#define AS_ERR_STATE       -6  /* key changed on a non-empty map, etc.      */
#define AS_ERR_UNSUPPORTED -7  /* configuration not built                   */
#define AS_ERR_CAPACITY    -8  /* entity map or arena full                  */
#define AS_ERR_AGAIN       -9  /* serving admission queue full: retry       */

/* Encoder arithmetic. FP32: FP32 everywhere (SIMT GEMM). BF16: GEMM inputs
 * rounded to BF16, FP32 accumulate; bias, residual, LayerNorm, softmax and
 * logits in FP32. FP8: GEMM inputs in E4M3 with static per-tensor scales
 * (weights: amax / 448 at as_create; activations: amax / 448 over a
 * calibration set, see as_calibrate), FP32 accumulate; Q/K/V and attention
 * in BF16/FP32; bias, residual, LayerNorm, softmax and logits in FP32. */
#define AS_FP32 0
#define AS_BF16 1
#define AS_FP8  2

/* Encoder batching. PACKED: all records of a call packed into large
 * variable-length batches. PER_RECORD: one record per launch sequence. */
#define AS_MODE_PACKED     0
#define AS_MODE_PER_RECORD 1

typedef struct as_ctx as_ctx;
typedef struct as_output as_output;

/* Model and runtime configuration, read by as_create only.
 * weights: host FP32 blob, n = weights_len floats, in this order (row-major,
 *   linear maps stored [out, in]):
 *     tok_emb[vocab][d], pos_emb[max_pos][d], emb_ln_g[d], emb_ln_b[d],
 *     per layer: w_qkv[3d][d] (rows 0..d-1 Q, d..2d-1 K, 2d..3d-1 V; head j
 *                owns rows j*dh..(j+1)*dh-1 of each), b_qkv[3d], w_o[d][d],
 *                b_o[d], ln1_g[d], ln1_b[d], w_1[f][d], b_1[f], w_2[d][f],
 *                b_2[d], ln2_g[d], ln2_b[d],
 *     cls_w[labels][d], cls_b[labels].
 * vocab: the strings of token ids 257..vocab-1 (ids 1..256 are single bytes
 *   0x00..0xFF, id 0 is padding): n_vocab_words = vocab - 257 strings of
 *   2..12 bytes from [0-9A-Za-z], string k at
 *   vocab_bytes[vocab_offsets[k] .. vocab_offsets[k+1]). Host memory. */
typedef struct {
  uint32_t vocab, d_model, n_heads, d_ffn, n_layers, n_labels, max_pos;
  uint32_t precision;            /* AS_FP32, AS_BF16 or AS_FP8                 */
  uint32_t mode;                 /* AS_MODE_PACKED or AS_MODE_PER_RECORD       */
  const float* weights;          /* host                                       */
  uint64_t weights_len;          /* floats                                     */
  const uint8_t* vocab_bytes;    /* host                                       */
  const uint32_t* vocab_offsets; /* host, n_vocab_words + 1 entries            */
  uint32_t n_vocab_words;
  uint64_t max_chunk_tokens;     /* encoder rows per packed batch; 0 = 1<<19   */
  uint64_t map_capacity;         /* entity-map slots (power of 2); 0 = 1<<22   */
  uint64_t map_arena_bytes;      /* bytes for map originals; 0 = 256 MiB       */
  int32_t device;                /* CUDA device ordinal                        */
  uint32_t keep_trace;           /* 1: keep per-stage results for as_debug_*   */
  uint32_t no_graphs;            /* 1: never replay CUDA graphs (see below)    */
  uint32_t attention;            /* BF16/FP8 attention engine: AS_ATTN_TCGEN05
                                    (0, default) or AS_ATTN_MMA_SYNC           */
  uint32_t no_fused_ln;          /* BF16/FP8 post-LN residual blocks run as one
                                    kernel (a row split over a cluster of CTAs;
                                    d_model 128, 256, 384, 512, 768 or 1024)
                                    unless set here as two kernels (GEMM, then
                                    LayerNorm): bit 0 the attention block,
                                    bit 1 the feed-forward block               */
} as_config;

/* Attention engines of BF16 and FP8 contexts: persistent tcgen05 kernel with
 * S, P and O in TMEM (default), or flash-style on mma.sync m16n8k16 tensor
 * cores (see include/anonshield_kernels.h). Results agree to BF16 rounding. */
#define AS_ATTN_TCGEN05  0
#define AS_ATTN_MMA_SYNC 1

/* Input records: one byte arena plus n_records + 1 offsets (offsets[0] = 0,
 * non-decreasing, offsets[n] = total bytes < 2^32). on_device = 0: host
 * pointers (copied to the GPU inside the call); 1: device pointers of the
 * ctx's device (read in place). */
typedef struct {
  const uint8_t* bytes;
  const uint64_t* offsets;
  uint64_t n_records;
  uint32_t on_device;
} as_records;

/* Pattern recognizers (AnonShield §2 stage (2) combines the NER model with
 * custom patterns for addresses, URLs, host names, hashes, certificates and
 * CVE/CPE identifiers; its entity types include UUIDs and OIDs). Index of a
 * recognizer in as_schema.recognizer_types. Word recognizers test one word
 * (a maximal run of [A-Za-z0-9.:-], trailing '.', '-', ':' stripped); the
 * multi-word ones (URL, CPE, PEM) start at a word start and may cover
 * several words. A candidate starting inside an accepted multi-word span is
 * dropped, as in a left-to-right regex scan. */
enum {
  AS_RX_MAC = 0,       /* six hex pairs joined by one of ':' '-'                     */
  AS_RX_IPV6 = 1,      /* 1..4-hex groups, eight, or at most seven with one '::'      */
  AS_RX_IPV4 = 2,      /* four octets 0..255, no leading zeros; ':port' not in span   */
  AS_RX_CVE = 3,       /* CVE-dddd-dddd+                                              */
  AS_RX_HOSTNAME = 4,  /* >= 2 labels, last one alphabetic; ':port' not in span       */
  AS_RX_URL = 5,       /* scheme://..., trailing .,:;!? stripped                      */
  AS_RX_HASH = 6,      /* 32, 40, 64 or 128 hex digits                                */
  AS_RX_UUID = 7,      /* 8-4-4-4-12 hex                                             */
  AS_RX_CPE = 8,       /* cpe:2.3: with 11 components, or cpe:/ URI form              */
  AS_RX_OID = 9,       /* >= 5 dotted decimal arcs, first 0..2                        */
  AS_RX_CERT_FP = 10,  /* 16, 20 or 32 hex pairs joined by ':'                        */
  AS_RX_PEM = 11,      /* -----BEGIN CERTIFICATE----- ... -----END CERTIFICATE-----   */
  AS_RX_KINDS = 12
};

/* Replacement policy. type_names[t-1] is the name of entity type t
 * (t = 1..n_types; label 2t-1 = B-t, 2t = I-t, 0 = O).
 * recognizer_types: NULL, or AS_RX_KINDS entries giving the entity type each
 * recognizer emits (0 = recognizer off; every type <= n_types). NULL maps
 * MAC to 4, IPv6 and IPv4 to 1, CVE to 3, host name to 2 (types 1
 * IP_ADDRESS, 2 HOSTNAME, 3 CVE_ID, 4 MAC_ADDRESS; needs n_types >= 4) and
 * switches the rest off. The table is copied by the call.
 * preserve_mask bit t set: type t is detected but passed through (the
 * paper's --entities-to-preserve, §2). slug_hex_len: 0..64 hex characters
 * (§2 stage (3)). window/stride: sliding windows for records longer than
 * window tokens (0 = none: a record over max_pos tokens is AS_ERR_TOO_LONG);
 * window <= max_pos, 0 < stride <= window, window - stride even. */
typedef struct {
  uint32_t n_types;
  const char* const* type_names;
  uint64_t preserve_mask;
  uint32_t slug_hex_len;
  uint32_t window, stride;
  const uint8_t* recognizer_types;
} as_schema;

/* One entity-map entry (§2 stage (4)): type, original bytes, full 64-hex
 * HMAC, slug, first / last record index, occurrences. */
typedef struct {
  uint32_t type;
  uint32_t original_len;
  const uint8_t* original;
  char full_hash[65];
  char slug[65];
  uint64_t first_seen, last_seen, count;
} as_entity;

/* Counters of one call. */
typedef struct {
  uint64_t n_records, n_bytes, n_tokens, n_encoded_tokens, n_sequences;
  uint64_t n_regex_spans, n_ner_spans, n_final_spans, n_out_bytes;
  uint64_t n_map_entries, n_new_entries;
  uint64_t kernel_launches;
  uint64_t graph_replays;        /* encoder batches run as one graph launch    */
  /* as_reidentify only: pseudonyms found, replaced by their originals, left
   * because several entries share the slug, left because the entry did not
   * verify under the key (the rest name no entry of the map) */
  uint64_t n_pseudonyms, n_reidentified, n_ambiguous, n_unverified;
  /* as_anonymize_jsonl only: fields found in the lines, lines that did not parse */
  uint64_t n_fields, n_malformed;
} as_stats;

/* Encoder batches of BF16 / FP8 contexts with the tcgen05 attention
 * (profiling off) run as one launch of a CUDA graph captured the first time
 * their shape bucket is seen (per lane; up to 16 buckets are kept). Rows and
 * attention work items are padded to the bucket: a power of two up to
 * AS_GRAPH_MAX_ROWS, above that the next multiple of 1/16 of the next power
 * of two (at most 6.25 % padding; full packed batches of the default 2^19-row
 * cap fill their bucket exactly, so every full batch of a call replays one
 * graph). Each batch's work items are copied into one fixed lane buffer
 * before the replay. Padded rows belong to no record and padded work items to
 * an empty sequence, so results are bit-identical to kernel-by-kernel
 * launches. The first encoder batch of a lane always runs kernel by kernel. */
#define AS_GRAPH_MAX_ROWS 16384

/* Create a context: loads weights and vocabulary onto `device`, creates the
 * ctx's stream. Errors: AS_ERR_ARG (shape mismatch, weights_len wrong,
 * vocab strings invalid), AS_ERR_UNSUPPORTED (d_model % 64 != 0 in BF16,
 * head dim != 64), AS_ERR_OOM, AS_ERR_CUDA. */
as_status as_create(const as_config* cfg, as_ctx** out);
void as_destroy(as_ctx* ctx);

/* Pseudonymise a batch. key: key_len bytes (RFC 2104; > 64 bytes is hashed
 * first). On success *out holds the output; free it with as_output_free.
 * Output records live on the host when records->on_device == 0, else on the
 * device. Errors: AS_ERR_ARG, AS_ERR_TOO_LONG, AS_ERR_STATE, AS_ERR_CAPACITY,
 * AS_ERR_TIMEOUT, AS_ERR_OOM, AS_ERR_CUDA. On error the map may hold entries
 * of records processed before the failure. */
as_status as_anonymize(as_ctx* ctx, const as_records* records, const as_schema* schema,
                       const uint8_t* key, size_t key_len, as_output** out);

/* Output records: arena + n+1 offsets; *on_device tells where they live. */
as_status as_output_records(const as_output* out, const uint8_t** bytes, const uint64_t** offsets,
                            uint64_t* n_records, uint32_t* on_device);
as_status as_output_stats(const as_output* out, as_stats* stats);
/* Map entries touched by this call (new or updated), sorted by (type, bytes).
 * Pointers valid until as_output_free; needs the ctx alive (as_output_records,
 * as_output_stats and as_output_free do not: an output may outlive its ctx). */
as_status as_output_map(as_output* out, const as_entity** entries, uint64_t* n);
void as_output_free(as_output* out);

/* The whole map, sorted by type, then original bytes (lexicographic, a
 * prefix first). *entries is one host allocation (entries followed by their
 * original bytes); free it with as_free. */
as_status as_map_export(as_ctx* ctx, as_entity** entries, uint64_t* n);
/* Load entries (e.g. a previous export, or another shard's map): an entry
 * already present keeps min first_seen, max last_seen, summed count. The
 * entries' full_hash must be the HMAC under this ctx's key. */
as_status as_map_import(as_ctx* ctx, const uint8_t* key, size_t key_len, const as_entity* entries, uint64_t n);
/* Union of the maps of replicas that processed disjoint record ranges of one
 * job (the one exchange of a multi-GPU run, done on the host; needs no GPU
 * and no ctx). shards[s] holds n[s] entries, e.g. that replica's export;
 * record_offset[s] (NULL = all 0) is the global index of that replica's
 * first record and is added to its first_seen / last_seen. Entries with the
 * same (type, original) keep min first_seen, max last_seen and the summed
 * count; their full_hash must agree (AS_ERR_STATE otherwise: the replicas
 * used different keys). The pseudonym being a function of key and bytes
 * alone (AnonShield §2 stage (4)), replicas never exchange anything else.
 * *out is sorted as in as_map_export, one allocation (free with as_free);
 * messages via as_last_error(NULL). */
as_status as_map_merge(const as_entity* const* shards, const uint64_t* n, const uint64_t* record_offset,
                       uint32_t n_shards, as_entity** out, uint64_t* n_out);
/* Empty the map and forget the key. */
as_status as_map_clear(as_ctx* ctx);

/* Per-stage results of the last as_anonymize (needs keep_trace = 1). Host
 * arrays owned by ctx, valid until the next call on ctx. Token arrays are in
 * record order: tok_ids/tok_off(byte offset in the batch arena)/tok_len, and
 * rec_tok[n+1] = first token of each record. Spans: start (byte offset in the
 * batch arena), length, type. logits: n_tokens x n_labels FP32 (window-merged).
 * labels: n_tokens. */
typedef struct {
  uint64_t n_records, n_tokens, n_regex, n_final;
  const uint64_t* rec_tok;
  const int32_t* tok_ids;
  const uint32_t* tok_off;
  const uint32_t* tok_len;
  const uint32_t* regex_start; const uint32_t* regex_len; const uint8_t* regex_type;
  const float* logits;
  const uint8_t* labels;
  const uint32_t* final_start; const uint32_t* final_len; const uint8_t* final_type;
} as_trace;
as_status as_debug_trace(as_ctx* ctx, as_trace* trace);

/* Controlled re-identification (AnonShield §2 stage (4): the stored mapping
 * lets an administrator holding both the database and the HMAC key reverse
 * the pseudonymisation). In `records` (same layout rules as as_anonymize),
 * every "[NAME_h]" inside one record, NAME = type_names[t-1] and h exactly
 * schema->slug_hex_len lower-case hex characters, is replaced by the original
 * bytes of the ctx's map entry of type t whose full hash begins with h, when
 * exactly one entry does and HMAC-SHA256(key, original) equals its full hash;
 * other bytes and unresolved pseudonyms are copied. Output in the inputs'
 * memory space, one record per input record; counts in as_stats
 * (n_pseudonyms, ...). Import a stored map with as_map_import first.
 * AS_ERR_ARG: slug_hex_len 0, or a type name containing '[' or ']';
 * AS_ERR_STATE: key differs from the non-empty map's key, or serving. */
as_status as_reidentify(as_ctx* ctx, const as_records* records, const as_schema* schema, const uint8_t* key,
                        size_t key_len, as_output** out);

/* Per-field policy: the schema-aware configuration of AnonShield §2
 * (anonymization_config with force_anonymize, fields_to_anonymize,
 * fields_to_exclude), which skips the detection steps for most of a record.
 * Each record holds fields: byte spans (start into the arena, length, field
 * id), sorted by start, disjoint, each inside one record. Per field id:
 *   AS_FIELD_DETECT   the field's bytes are a record of their own for every
 *                     detection step (tokenizer, recognizers, encoder with
 *                     windows, BIO decode, overlap rule, preserve list); the
 *                     spans found are shifted by the field start;
 *   AS_FIELD_EXCLUDE  the field passes through unchanged (never scanned);
 *   AS_FIELD_FORCE    the field's value, ASCII whitespace trimmed at both ends,
 *                     is one entity of force_type (1..n_types), replaced
 *                     whatever the preserve list says; nothing if empty.
 * Bytes outside every field (separators, keys, layout) pass through
 * unchanged. Ids >= n_ids take default_action (DETECT or EXCLUDE). Record
 * indices, map and output are those of the records. Fields and policy are
 * host arrays; records may be on the host or the device (as_anonymize). The
 * debug trace's token arrays then describe the arena of detected fields (one
 * sub-record per field, in field order). Errors as as_anonymize, plus
 * AS_ERR_ARG for unsorted, overlapping or record-crossing fields and invalid
 * actions or types. */
#define AS_FIELD_DETECT  0
#define AS_FIELD_EXCLUDE 1
#define AS_FIELD_FORCE   2
typedef struct {
  const uint64_t* start;   /* byte offset of each field in the arena        */
  const uint32_t* len;
  const uint32_t* id;      /* field id (column or key index)                */
  uint64_t n_fields;
} as_fields;
typedef struct {
  uint32_t n_ids;
  const uint8_t* action;      /* per field id: AS_FIELD_*                     */
  const uint8_t* force_type;  /* per field id: entity type for AS_FIELD_FORCE */
  uint8_t default_action;     /* for ids >= n_ids                             */
} as_field_policy;
as_status as_anonymize_fields(as_ctx* ctx, const as_records* records, const as_fields* fields,
                              const as_field_policy* policy, const as_schema* schema, const uint8_t* key,
                              size_t key_len, as_output** out);

/* JSON Lines ingest (AnonShield §2: JSON / JSONL inputs keep their structure,
 * only sensitive values are replaced, with per-field control). Each record is
 * one line (no newline). On the device, a line that is one JSON value
 * (RFC 8259; white space around it; at most 64 nested containers; strings
 * without raw bytes below 0x20, escapes \" \\ \/ \b \f \n \r \t \uXXXX)
 * yields one field per run of a string VALUE's raw bytes outside escape
 * sequences, so replacements keep the line valid JSON; member keys, numbers,
 * literals and punctuation are structure and pass through. A field's action
 * is that of its innermost enclosing member key (key_names compared as raw
 * bytes): action[i] / force_type[i] for key_names[i], default_action for
 * other keys and for values in no member. A line that does not parse is
 * detected as free text as a whole (never passed through unchanged); an
 * empty line has no fields. Then as for as_anonymize_fields. Stats:
 * n_fields, n_malformed. */
typedef struct {
  uint32_t n_keys;
  const char* const* key_names;
  const uint8_t* action;       /* per key: AS_FIELD_*                          */
  const uint8_t* force_type;   /* per key: entity type for AS_FIELD_FORCE      */
  uint8_t default_action;      /* AS_FIELD_DETECT or AS_FIELD_EXCLUDE          */
} as_jsonl_policy;
as_status as_anonymize_jsonl(as_ctx* ctx, const as_records* records, const as_jsonl_policy* policy,
                             const as_schema* schema, const uint8_t* key, size_t key_len, as_output** out);

/* Streaming (AnonShield §2 stage (1) reads large inputs as a stream): the
 * same result as one as_anonymize call over `records` (host memory only),
 * computed in consecutive batches of at most batch_bytes (a longer record
 * goes alone). `lanes` worker threads each own a CUDA stream, device buffers
 * and a pinned staging buffer: a worker copies its batch into pinned memory,
 * the H2D copy, kernels and D2H of one batch overlap those of the others.
 * Record indices are positions in `records` (plus earlier calls), so the
 * output bytes and the map equal those of a single call. The output is on
 * the host; as_output_map gives the entries touched by this call. Errors as
 * as_anonymize (the message names the failing batch); on error, batches
 * that completed have updated the map. */
typedef struct {
  uint64_t batch_bytes;  /* 0 = 16 MiB */
  uint32_t lanes;        /* concurrent batches, 0 = 2 (max 8) */
} as_stream_config;
as_status as_anonymize_stream(as_ctx* ctx, const as_records* records, const as_schema* schema, const uint8_t* key,
                              size_t key_len, const as_stream_config* cfg, as_output** out);

/* Serving loop (continuous batching). After as_serve_start the ctx accepts
 * single records with as_submit from any thread; worker threads (one per
 * lane, each with its own CUDA stream and buffers) take the oldest waiting
 * requests, run the whole path on them and post the results; with two or
 * more lanes a batch starts while others are still on the GPU.
 *
 * Admission is by device memory: activation_budget_bytes bounds the encoder
 * activations of all lanes together (a 1/lanes share each). A lane's share
 * fixes its row cap R: the most encoder rows whose activation buffers (per
 * row: the FP32 residual and pre-LN rows, the BF16 / E4M3 GEMM inputs, QKV,
 * attention output and FFN rows, row indices; padded to the graph bucket,
 * each buffer allocated with 1/8 slack) fit the share. A worker admits the oldest requests while the
 * rows they can occupy at most (a record of b bytes has at most b tokens;
 * windows and the 8-row alignment added) stay within R; the first request is
 * always admitted, and encoder batches never exceed R rows (a long record
 * runs as several), so a lane's activation buffers stay within its share.
 * max_batch_bytes and max_batch_records are further caps (0 = none / 65536).
 * as_serve_start fails with AS_ERR_ARG if a share cannot hold one full
 * sequence (max_pos rows).
 *
 * A request's record index (first_seen / last_seen) is its request id, and
 * every step computes a record from that record's data alone, so the result
 * of a request is the same alone and in any mix. The entity map stays on the
 * device; as_map_export gives a snapshot. as_anonymize and as_calibrate
 * return AS_ERR_STATE while serving. */
typedef struct {
  uint32_t lanes;              /* concurrent batches on the GPU; 0 = 2        */
  uint64_t max_batch_bytes;    /* record bytes per batch; 0 = no byte cap     */
  uint32_t max_batch_records;  /* 0 = 65536                                    */
  uint64_t max_pending;        /* queue bound (AS_ERR_AGAIN beyond); 0 = 2^20 */
  uint64_t activation_budget_bytes; /* encoder activations, all lanes; 0 = 40 GiB */
} as_serve_config;
typedef struct {
  uint64_t completed, rejected, failed, batches, tokens, pending;
  double seconds;              /* since start or the last reset               */
  double p50_ms, p99_ms, max_ms; /* submit -> result ready, completed requests */
  uint64_t activation_budget;  /* bytes, all lanes                            */
  uint64_t row_cap;            /* encoder rows per batch and lane             */
  uint64_t activation_bytes;   /* activation buffers the lanes hold now       */
  uint64_t activation_peak;    /* the most they held at once since start      */
} as_serve_stats_t;
#define AS_SUBMIT_DISCARD 1u   /* drop the result (load tests): latency only  */
as_status as_serve_start(as_ctx* ctx, const as_schema* schema, const uint8_t* key, size_t key_len,
                         const as_serve_config* cfg);
/* Copy one record and queue it; *request_id identifies it for as_poll.
 * AS_ERR_AGAIN when max_pending requests are already waiting. */
as_status as_submit(as_ctx* ctx, const uint8_t* record, uint64_t len, uint32_t flags, uint64_t* request_id);
/* Wait up to timeout_us for a request; on success *out holds its one output
 * record (host memory; free with as_output_free). AS_ERR_TIMEOUT leaves the
 * request queued; a finished request can be polled once. */
as_status as_poll(as_ctx* ctx, uint64_t request_id, as_output** out, int64_t timeout_us);
/* Counters and latency percentiles; reset = 1 starts a new window. */
as_status as_serve_stats(as_ctx* ctx, as_serve_stats_t* stats, uint32_t reset);
/* Finish every admitted request, then stop the workers. */
as_status as_serve_stop(as_ctx* ctx);

/* Tile autotuner for the encoder's four tcgen05 projection GEMMs (per
 * layer: QKV, attention output + residual, FFN1 + GELU, FFN2 + residual).
 * Configurations: bit 0 = tile order (0: along N within a 128-row block,
 * 1: along M within a column block), bit 1 = 128-column tiles with 6
 * pipeline stages instead of 256-column tiles with 4 (configurations
 * without bit 1 need N % 256 == 0), bit 2 = 2-SM pairs (a cluster of two
 * CTAs computing one 256-row tile with cta_group::2 MMAs; each CTA loads its
 * own 128 A rows and half of the weight tile, no multicast); -1 = the built-in
 * default (cfg 0 when valid, else 2). A post-LN block run as one fused
 * kernel (roles 1 and 3, see as_config.no_fused_ln) has four choices: cfg 0
 * (single-CTA tiles), 4 (2-SM pairs), and each | 2 (a shorter main-loop ring
 * for more residual / output bytes in flight in the epilogue); its default is
 * 0 for role 1 and 4 for role 3; odd configurations report ms < 0.
 * as_autotune times every valid configuration of each projection at `rows`
 * rows (0 = the ctx's batch size, max_chunk_tokens) on the ctx's stream with
 * the ctx's weights and scratch activations, keeps the fastest for later
 * calls and reports all timings (ms < 0: not valid). Results do not depend on
 * the configuration (the tile only changes which CTA computes an output).
 * AS_ERR_UNSUPPORTED for FP32 contexts (CUDA-core GEMM). as_set_tiles /
 * as_get_tiles store or read the choices, e.g. to reuse a saved tuning. */
#define AS_TUNE_ROLES 4
#define AS_TUNE_CONFIGS 8
typedef struct {
  uint32_t role;       /* 0 QKV, 1 attention output, 2 FFN1, 3 FFN2        */
  uint64_t m, n, k;
  int32_t chosen;
  float ms[AS_TUNE_CONFIGS]; /* per configuration; negative = not valid    */
} as_tune_entry;
as_status as_autotune(as_ctx* ctx, uint64_t rows, as_tune_entry entries[AS_TUNE_ROLES]);
as_status as_set_tiles(as_ctx* ctx, const int32_t cfg[AS_TUNE_ROLES]);
as_status as_get_tiles(as_ctx* ctx, int32_t cfg[AS_TUNE_ROLES]);

/* FP8 contexts: set the static activation scales from a calibration set.
 * Runs the tokenizer and the BF16 encoder over `records` (same layout rules
 * as as_anonymize) and records, for each FP8 GEMM input (per layer: the QKV,
 * output, FFN-in and FFN-out projection inputs), the largest magnitude; each
 * scale is that amax / 448 (the E4M3 maximum). Fixed scales make a record's
 * result independent of the batch it arrives in. Touches neither the map nor
 * the key. Errors: AS_ERR_STATE (not an FP8 context), as as_anonymize. */
as_status as_calibrate(as_ctx* ctx, const as_records* records, const as_schema* schema);
/* Read / load the activation scales (4 per layer, order above) so that a
 * calibration can be stored with the weights and reused. */
as_status as_get_scales(as_ctx* ctx, float* scales, uint64_t n);
as_status as_set_scales(as_ctx* ctx, const float* scales, uint64_t n);

/* The ctx's CUDA stream (a cudaStream_t): every kernel of the ctx runs on
 * it, so a caller can time a call with CUDA events recorded on it. */
as_status as_get_stream(as_ctx* ctx, void** stream);

/* Opt-in launch timing. enable = 1 records a CUDA event pair around every
 * encoder GEMM and attention launch of later calls and accumulates their
 * device time and algorithmic FLOPs (GEMM 2*M*N*K; attention 4*L^2*d per
 * sequence of L tokens); enable = 0 stops and clears. Timing adds a few
 * microseconds per launch. The integer stages of the ctx's own batch calls
 * (as_anonymize, as_anonymize_fields, as_anonymize_jsonl) are timed the same
 * way, one event pair around each stage's launches (host syncs and output
 * allocation excluded): stage_ms[0] tokenizer + recognizers (§2 stage (2)
 * patterns), [1] BIO decode, overlap rule, preserve list and span merge,
 * [2] HMAC-SHA256 + entity-map upsert (§2 stages (3), (4)), [3] substitution
 * (replacement lengths, output shifts, pass-through copy, pseudonym writes,
 * output offsets; §2 stage (5)); stage_calls counts the timed calls. */
typedef struct {
  uint64_t gemm_launches;
  double gemm_ms, gemm_flops;
  uint64_t attn_launches;
  double attn_ms, attn_flops;
  uint64_t stage_calls;
  double stage_ms[4];
} as_profile_stats;
as_status as_profile(as_ctx* ctx, uint32_t enable);
as_status as_profile_read(as_ctx* ctx, as_profile_stats* stats);

/* Tokenizer that allocates no memory. The paper has no counterpart: this is
 * for callers that cannot call cudaMalloc, such as hosts whose device memory
 * belongs to their own allocator (reserved up front and handed out by the
 * host itself), or latency-bound loops where an allocation would synchronize
 * the device and stall work already queued on it. It runs the same tokenizer
 * as as_anonymize, with its scratch memory in a fixed-size array inside the
 * library instead of ctx buffers.
 * All pointers are device pointers on the ctx's device:
 *   bytes[n_bytes], offsets[n_records + 1] (offsets[n_records] == n_bytes),
 *   outputs tok_ids / tok_off (byte offset in `bytes`) / tok_len with room
 *   for n_bytes tokens, rec_tok[n_records + 1] (first token of each record),
 *   *n_tokens (token count).
 * Asynchronous on `stream` (a cudaStream_t; NULL = legacy default stream).
 * Limits: n_bytes <= AS_STATIC_MAX_BYTES, else AS_ERR_ARG. The array (about
 * 6.4 MB) stays on every device that loads the library until exit. The first
 * call on a device looks the array up (cudaGetSymbolAddress): make it before
 * any stream capture. Every call reuses the same array, so calls that overlap
 * on the GPU (other streams or host threads) race: serialize them. The call
 * makes the ctx's device current while it runs and restores the caller's
 * current device before returning. */
#define AS_STATIC_MAX_BYTES (1u << 20)
as_status as_tokenize_static(as_ctx* ctx, const uint8_t* bytes, const uint64_t* offsets, uint64_t n_records,
                             uint64_t n_bytes, int32_t* tok_ids, uint32_t* tok_off, uint32_t* tok_len,
                             uint64_t* rec_tok, uint32_t* n_tokens, void* stream);

const char* as_last_error(const as_ctx* ctx);
void as_free(void* p);
/* Library version string. */
const char* as_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ANONSHIELD_H */
