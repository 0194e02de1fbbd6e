// Declarations of the batch stages (tokenizer, recognizers, BIO decode,
// span merge, HMAC, entity map, substitution) launched by the runtime.
#pragma once

#include "common.cuh"

namespace as {

// ---- vocabulary hash table (greedy longest-match lookups) ----
// A slot holds up to 12 bytes packed little-endian in x, y, z and
// w = length | id << 16 (w == 0: empty). Open addressing, linear probing.
constexpr int kMaxPiece = 12;

__host__ __device__ inline uint32_t vocab_hash(uint32_t w0, uint32_t w1, uint32_t w2, uint32_t len) {
  uint32_t h = len * 0x9E3779B1u;
  h ^= w0; h *= 0x85EBCA77u; h ^= h >> 13;
  h ^= w1; h *= 0xC2B2AE3Du; h ^= h >> 16;
  h ^= w2; h *= 0x27D4EB2Fu; h ^= h >> 15;
  return h;
}

// Open-addressing table of the vocabulary strings (slot = the string's
// bytes in x,y,z and len | id << 16 in w; w == 0 marks an empty slot), and
// for each pair of leading alphanumeric bytes the set of vocabulary lengths
// that start with that pair (bit L set: some string of length L does), so
// the greedy match probes only lengths that can hit.
constexpr int kAlnumCodes = 62;
__host__ __device__ inline uint32_t alnum_code(uint32_t c) {
  return c <= '9' ? c - '0' : c <= 'Z' ? c - 'A' + 10 : c - 'a' + 36;
}
struct VocabTable {
  const uint4* slots;
  uint32_t mask;
  const uint16_t* lenmask;  // [kAlnumCodes * kAlnumCodes]
};

// ---- stage launchers (all asynchronous on `st`) ----
// Bit r of the bitmap is set when a record starts at byte r (n_words = N/32 + 1).
void launch_mark_record_starts(const uint64_t* offsets, uint64_t n_records, uint32_t N, uint32_t* rs_bits,
                               cudaStream_t st);
// tok_at[i] = token id when a token starts at byte i, else 0. With
// tile_sums (scan_tiles_needed(N) elements, zeroed by the caller), also the
// number of token starts in each 4,096-byte tile.
void launch_tokenize_mark(const uint8_t* bytes, uint32_t N, const uint32_t* rs_bits, VocabTable vt,
                          uint16_t* tok_at, cudaStream_t st, uint32_t* tile_sums = nullptr);
// Compact token starts: ids/offsets in byte order; pos[] is the exclusive scan.
void launch_tokenize_emit(const uint16_t* tok_at, const uint32_t* pos, uint32_t N, int32_t* tok_ids,
                          uint32_t* tok_off, cudaStream_t st);
void launch_token_lengths(const uint32_t* tok_off, uint32_t T, uint32_t N, uint32_t* tok_len, cudaStream_t st);
void launch_record_token_offsets(const uint64_t* offsets, uint64_t n_records, const uint32_t* pos, uint32_t N,
                                 const uint32_t* total_T, uint64_t* rec_tok, cudaStream_t st);
// Token table (id, first byte) in byte order from the marks; *n_tokens = T.
// tile_scratch: scan_tiles_needed(N) elements.
void launch_tokenize_compact(const uint16_t* tok_at, uint32_t N, int32_t* ids, uint32_t* off, uint32_t* n_tokens,
                             uint32_t* tile_scratch, cudaStream_t st);
// The same table plus token lengths, from the tile counts that
// launch_tokenize_mark wrote into tile_sums (turned into tile offsets here).
void launch_tokenize_table(const uint16_t* tok_at, uint32_t N, int32_t* ids, uint32_t* off, uint32_t* len,
                           uint32_t* n_tokens, uint32_t* tile_sums, cudaStream_t st);
// rec_tok[r] = first token of record r (T for offsets at N), from the token offsets.
void launch_record_token_starts(const uint64_t* offsets, uint64_t n, const uint32_t* tok_off, const uint32_t* total_T,
                                uint32_t N, uint64_t* rec_tok, cudaStream_t st);

// Pattern recognizers: rx_len[i] / rx_type[i] at each word start that is an
// entity candidate. RxTypes maps each recognizer kind (the order of
// as_rx_kind: MAC, IPv6, IPv4, CVE, host name, URL, hash, UUID, CPE, OID,
// certificate fingerprint, PEM certificate) to an entity type, 0 = off.
// Candidates of the multi-word kinds (URL, CPE, PEM) carry kRxLong in their
// type until launch_recognize_resolve has dropped every candidate that starts
// inside an accepted multi-word span; it must run whenever one of those
// kinds is on.
constexpr int kRxMac = 0, kRxIpv6 = 1, kRxIpv4 = 2, kRxCve = 3, kRxHost = 4, kRxUrl = 5, kRxHash = 6, kRxUuid = 7,
              kRxCpe = 8, kRxOid = 9, kRxCertFp = 10, kRxPem = 11, kRxKinds = 12;
constexpr uint8_t kRxLong = 0x80;
struct RxTypes {
  uint8_t t[kRxKinds];
};
inline bool rx_any_long(const RxTypes& r) { return r.t[kRxUrl] || r.t[kRxCpe] || r.t[kRxPem]; }
// rx_type[i] for every byte (0: no candidate starts there); rx_len[i] only
// where rx_type[i] != 0. tile_sums as for launch_tokenize_mark (candidates).
void launch_recognize_mark(const uint8_t* bytes, uint32_t N, const uint32_t* rs_bits, RxTypes types,
                           uint32_t* rx_len, uint8_t* rx_type, cudaStream_t st, uint32_t* tile_sums = nullptr);
void launch_recognize_resolve(const uint64_t* offsets, uint64_t n_records, const uint32_t* rx_len, uint8_t* rx_type,
                              cudaStream_t st);
// Recognizer spans (start, length, type) in byte order; *n_spans = their count.
void launch_recognize_compact(const uint32_t* rx_len, const uint8_t* rx_type, uint32_t N, uint32_t* sp_start,
                              uint32_t* sp_len, uint8_t* sp_type, uint32_t* n_spans, uint32_t* tile_scratch,
                              cudaStream_t st, bool sums_given = false);

// BIO decode: token flags (bit0 first token of record, bit1 last).
void launch_token_flags(const uint64_t* rec_tok, uint64_t n_records, uint8_t* tok_flags, cudaStream_t st);
// start[t] = 1 when a span starts at token t; is_end[t] = 1 when one ends there.
void launch_bio_mark(const uint8_t* labels, const uint8_t* tok_flags, uint32_t T, uint8_t* is_start,
                     uint8_t* is_end, cudaStream_t st);
// Token spans: ner_start / ner_len receive the first / last token of each span.
void launch_bio_emit(const uint8_t* labels, const uint8_t* is_start, const uint8_t* is_end, const uint32_t* pos,
                     uint32_t T, const uint32_t* tok_off, const uint32_t* tok_len, const uint8_t* bytes,
                     uint32_t* ner_start, uint32_t* ner_len, uint8_t* ner_type, cudaStream_t st);
// In place: (first token, last token) -> trimmed byte span (length 0 = dropped).
void launch_bio_to_bytes(uint32_t* ner_start, uint32_t* ner_len, const uint32_t* n_dev, uint32_t cap,
                         const uint32_t* tok_off, const uint32_t* tok_len, const uint8_t* bytes, cudaStream_t st);
// keep[k] for NER spans: non-empty, not overlapping any recognizer span, type not preserved.
void launch_ner_keep(const uint32_t* ner_start, const uint32_t* ner_len, const uint8_t* ner_type,
                     const uint32_t* n_ner_dev, uint32_t ner_cap, const uint32_t* rx_start, const uint32_t* rx_len,
                     const uint32_t* n_rx_dev, uint64_t preserve_mask, uint8_t* keep, cudaStream_t st);
void launch_rx_keep(const uint8_t* rx_type, const uint32_t* n_rx_dev, uint32_t rx_cap, uint64_t preserve_mask,
                    uint8_t* keep, cudaStream_t st);
// Compact a span list by keep[] (pos = exclusive scan of keep).
void launch_compact_spans(const uint32_t* s, const uint32_t* l, const uint8_t* t, const uint8_t* keep,
                          const uint32_t* pos, const uint32_t* n_dev, uint32_t cap, uint32_t* os, uint32_t* ol,
                          uint8_t* ot, cudaStream_t st);
// Merge two sorted disjoint lists into one sorted list.
void launch_merge_spans(const uint32_t* a_s, const uint32_t* a_l, const uint8_t* a_t, const uint32_t* n_a_dev,
                        uint32_t a_cap, const uint32_t* b_s, const uint32_t* b_l, const uint8_t* b_t,
                        const uint32_t* n_b_dev, uint32_t b_cap, uint32_t* o_s, uint32_t* o_l, uint8_t* o_t,
                        cudaStream_t st);

// ---- per-field policy (fields.cu) ----
// Copy detected fields to their sub-records (sub_off: nf + 1 offsets).
void launch_field_gather(const uint8_t* bytes, const uint32_t* f_start, const uint64_t* sub_off, uint64_t nf,
                         uint8_t* sub, cudaStream_t st);
// Trim forced spans in place; keep[i] = non-empty.
void launch_field_force_trim(const uint8_t* bytes, uint32_t* s, uint32_t* l, uint8_t* keep, uint32_t n,
                             cudaStream_t st);
// Sub-record span starts -> record coordinates.
void launch_field_translate(uint32_t* sp_s, const uint32_t* n_dev, uint32_t cap, const uint64_t* sub_off, uint64_t nf,
                            const uint32_t* f_start, cudaStream_t st);
// *dst += *add (device counters).
void launch_add_count(uint32_t* dst, const uint32_t* add, cudaStream_t st);

// ---- HMAC-SHA256 ----
void sha256_init_constants();  // uploads FIPS 180-4 constants (derived on the host)
// key_state[0..7] = inner midstate, [8..15] = outer midstate.
void launch_hmac_key_setup(const uint8_t* key, uint32_t key_len, uint32_t* key_state, cudaStream_t st);
void launch_hmac_spans(const uint8_t* bytes, const uint32_t* sp_start, const uint32_t* sp_len,
                       const uint32_t* n_dev, uint32_t cap, const uint32_t* key_state, uint32_t* digests,
                       cudaStream_t st);

// ---- entity map ----
struct MapSlot {
  unsigned long long key;         // 0 = empty; type << 56 | 56 bits of the digest
  unsigned long long first_seen;  // atomicMin
  unsigned long long last_seen;   // atomicMax
  unsigned long long count;       // atomicAdd
  uint32_t digest[8];             // full HMAC (written by the inserting thread)
  unsigned long long arena_off;   // original bytes in the arena
  uint32_t len;
  uint32_t type;
  uint32_t first_call;            // call id that created the entry
  uint32_t last_call;             // atomicMax of call ids that touched it
};
struct MapView {
  MapSlot* slots;
  uint64_t mask;
  uint8_t* arena;
  unsigned long long* arena_used;
  uint64_t arena_cap;
  unsigned long long* n_entries;
};
void launch_map_init(MapView m, cudaStream_t st);
// Insert/update one entry per final span; record index = rec_base + record of the span.
void launch_map_insert_spans(MapView m, const uint8_t* bytes, const uint32_t* sp_start, const uint32_t* sp_len,
                             const uint8_t* sp_type, const uint32_t* digests, const uint32_t* n_dev, uint32_t cap,
                             const uint64_t* offsets, uint64_t n_records, uint64_t rec_base, uint32_t call_id,
                             DevError* err, cudaStream_t st);
// Import entries (host-prepared arrays already on the device).
void launch_map_import(MapView m, const uint8_t* orig, const uint64_t* orig_off, const uint32_t* orig_len,
                       const uint32_t* type, const uint32_t* digests, const uint64_t* first, const uint64_t* last,
                       const uint64_t* count, uint64_t n, uint32_t call_id, DevError* err, cudaStream_t st);
// keep[i] = slot i occupied and (call_id == 0 or touched by call_id).
// keep[i] = slot i holds an entry last touched by a call in [call_lo, call_hi]
// (call_lo = 0: every entry).
void launch_map_select(MapView m, uint32_t call_lo, uint32_t call_hi, uint8_t* keep, cudaStream_t st);
void launch_map_gather(MapView m, const uint8_t* keep, const uint32_t* pos, uint32_t* idx, cudaStream_t st);
void launch_map_gather_slots(MapView m, const uint32_t* idx, uint32_t n, MapSlot* out, cudaStream_t st);

// ---- JSON Lines ingest ----
constexpr int kJsonMaxDepth = 64;
struct JsonKeys {
  const char* names;    // key i = names[off[i] .. off[i+1])
  const uint32_t* off;
  uint32_t n;
};
// cnt[r] = fields of line r (1 for a malformed line, bad[r] = 1, *n_bad += 1).
void launch_jsonl_count(const uint8_t* bytes, const uint64_t* off, uint64_t n, JsonKeys K, uint32_t* cnt, uint8_t* bad,
                        unsigned long long* n_bad, cudaStream_t st);
// Writes line r's fields at pos[r] (exclusive prefix sum of cnt).
void launch_jsonl_emit(const uint8_t* bytes, const uint64_t* off, uint64_t n, JsonKeys K, const uint32_t* pos,
                       const uint8_t* bad, uint64_t* f_start, uint32_t* f_len, uint32_t* f_id, cudaStream_t st);

// ---- re-identification ----
// ok[i] = 1: map slot i holds an entry whose digest is the HMAC of its original.
void launch_hmac_verify_slots(MapView m, const uint32_t* key_state, uint8_t* ok, cudaStream_t st);
// (type, slug prefix) -> map slot index; key 0 = empty.
constexpr uint32_t kReidEmpty = 0xffffffffu, kReidAmbiguous = 0xfffffffeu;
struct ReidTab {
  unsigned long long* key;
  uint32_t* val;
  uint64_t mask;
};
void launch_reid_index(MapView m, uint32_t p_bits, ReidTab tab, cudaStream_t st);
void launch_reid_mark(const uint8_t* bytes, uint32_t N, const uint32_t* rs_bits, const char* names,
                      const uint32_t* name_off, uint32_t n_types, uint32_t slug_len, ReidTab tab, MapView m,
                      const uint8_t* ok, uint32_t* plen, uint32_t* pslot, uint8_t* flag, unsigned long long* ctr,
                      cudaStream_t st);
void launch_reid_emit(const uint32_t* plen, const uint32_t* pslot, const uint8_t* flag, const uint32_t* pos, uint32_t N,
                      uint32_t* sp_s, uint32_t* sp_l, uint32_t* sp_k, cudaStream_t st);
void launch_reid_delta(const uint32_t* sp_l, const uint32_t* sp_k, uint32_t n, MapView m, int64_t* delta, uint32_t cap,
                       cudaStream_t st);
void launch_reid_replace(const uint32_t* sp_s, const uint32_t* sp_k, uint32_t n, const int64_t* shift, MapView m,
                         uint8_t* out, cudaStream_t st);

// ---- substitution ----
// delta[k] = replacement length - span length (int64).
void launch_sub_delta(const uint32_t* sp_len, const uint8_t* sp_type, const uint32_t* n_dev, uint32_t cap,
                      const uint32_t* name_len, uint32_t slug_len, int64_t* delta, cudaStream_t st);
void launch_sub_copy(const uint8_t* bytes, uint32_t N, const uint32_t* sp_start, const uint32_t* sp_len,
                     const uint32_t* n_dev, const int64_t* shift, uint8_t* out, cudaStream_t st);
void launch_sub_replace(const uint32_t* sp_start, const uint8_t* sp_type, const uint32_t* n_dev, uint32_t cap,
                        const int64_t* shift, const uint32_t* digests, const char* names, const uint32_t* name_off,
                        uint32_t slug_len, uint8_t* out, cudaStream_t st);
void launch_sub_offsets(const uint64_t* offsets, uint64_t n_records, const uint32_t* sp_start,
                        const uint32_t* n_dev, const int64_t* shift, uint64_t* out_off, cudaStream_t st);

}  // namespace as
