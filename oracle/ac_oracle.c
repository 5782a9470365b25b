/*
 * ac_oracle.c -- serial CPU Aho-Corasick pattern matching machine.
 *
 * TEST INFRASTRUCTURE, NOT PART OF THE LIBRARY.  Only the test suite, the
 * package smoke check and the benchmark's CPU-baseline leg may load this
 * code.  It shares nothing with the CUDA path: no headers, no tables, no
 * helpers.
 *
 * What it follows (paper section II): a finite-state pattern matching
 * machine built from the keyword set, with three functions --
 *   goto    : the trie of the keywords (child reached from a state on a byte),
 *   failure : the state to fall back to when goto has no edge,
 *   output  : the keywords recognised on entering a state,
 * and one serial pass over the text, character by character (section I,
 * Fig. 3), that emits every (end position, keyword id) occurrence.
 *
 * The failureless (PFAC) machine reports, for every start position, only
 * the longest keyword beginning there; it drops the sub-pattern outputs
 * (section II).  This file reaches that result by a different route: the
 * full machine's (end, id) occurrences are converted to start positions
 * and, per start, the longest keyword is kept (equal strings: lowest id).
 *
 * Plain data structures on purpose: every state keeps its goto edges as a
 * singly linked list of children, like the CPU machine of Fig. 4.  Nothing
 * here is tuned.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    int32_t first_child;  /* head of this state's goto-edge list, -1 if none   */
    int32_t next_sibling; /* next edge in the parent's list, -1 at the end      */
    int32_t fail;         /* failure function                                   */
    int32_t dict;         /* nearest state on the failure chain (excluding this
                             one) whose own keyword list is non-empty, or -1    */
    int32_t own_head;     /* first keyword id that ends exactly here, or -1     */
    int32_t own_tail;     /* last keyword id of that list, or -1                */
    int32_t depth;        /* length of the string spelled from the root         */
    uint8_t byte;         /* label of the goto edge that enters this state      */
} oracle_node;

typedef struct {
    oracle_node *nodes;
    uint32_t n_nodes;
    uint32_t cap;
    uint32_t k;           /* number of keywords                                 */
    uint64_t *klen;       /* length of each keyword                             */
    int32_t *own_next;    /* own_next[id]: next keyword id in the same state    */
} oracle_ac;

/* goto(s, a): the child of s on byte a, or -1 when the edge is missing. */
static int32_t oracle_goto(const oracle_ac *m, int32_t s, uint8_t a)
{
    int32_t c = m->nodes[s].first_child;
    while (c >= 0) {
        if (m->nodes[c].byte == a) return c;
        c = m->nodes[c].next_sibling;
    }
    return -1;
}

static int32_t oracle_new_node(oracle_ac *m, int32_t parent, uint8_t a)
{
    if (m->n_nodes == m->cap) {
        uint32_t cap = m->cap ? 2 * m->cap : 1024;
        oracle_node *p = (oracle_node *)realloc(m->nodes, (size_t)cap * sizeof(oracle_node));
        if (!p) return -1;
        m->nodes = p;
        m->cap = cap;
    }
    int32_t id = (int32_t)m->n_nodes++;
    oracle_node *x = &m->nodes[id];
    x->first_child = -1;
    x->next_sibling = -1;
    x->fail = 0;
    x->dict = -1;
    x->own_head = -1;
    x->own_tail = -1;
    x->byte = a;
    x->depth = 0;
    if (parent >= 0) {
        x->depth = m->nodes[parent].depth + 1;
        x->next_sibling = m->nodes[parent].first_child;
        m->nodes[parent].first_child = id;
    }
    return id;
}

void oracle_ac_free(oracle_ac *m)
{
    if (!m) return;
    free(m->nodes);
    free(m->klen);
    free(m->own_next);
    free(m);
}

/*
 * Build the machine.  Keyword i is bytes[off[i] .. off[i+1]).  Empty keywords
 * are refused (returns NULL), as is k == 0.
 */
oracle_ac *oracle_ac_build(const uint8_t *bytes, const uint64_t *off, uint32_t k)
{
    if (k == 0) return NULL;
    oracle_ac *m = (oracle_ac *)calloc(1, sizeof(oracle_ac));
    if (!m) return NULL;
    m->k = k;
    m->klen = (uint64_t *)malloc((size_t)k * sizeof(uint64_t));
    m->own_next = (int32_t *)malloc((size_t)k * sizeof(int32_t));
    if (!m->klen || !m->own_next || oracle_new_node(m, -1, 0) != 0) {
        oracle_ac_free(m);
        return NULL;
    }

    /* goto function: insert every keyword into the trie. */
    for (uint32_t id = 0; id < k; ++id) {
        uint64_t len = off[id + 1] - off[id];
        if (len == 0) {
            oracle_ac_free(m);
            return NULL;
        }
        m->klen[id] = len;
        m->own_next[id] = -1;
        int32_t s = 0;
        for (uint64_t j = 0; j < len; ++j) {
            uint8_t a = bytes[off[id] + j];
            int32_t t = oracle_goto(m, s, a);
            if (t < 0) {
                t = oracle_new_node(m, s, a);
                if (t < 0) {
                    oracle_ac_free(m);
                    return NULL;
                }
            }
            s = t;
        }
        /* output function, own part: the keyword ends at state s.  Ids are
           appended in increasing order. */
        if (m->nodes[s].own_head < 0) {
            m->nodes[s].own_head = (int32_t)id;
        } else {
            m->own_next[m->nodes[s].own_tail] = (int32_t)id;
        }
        m->nodes[s].own_tail = (int32_t)id;
    }

    /* failure function, breadth first: a depth-1 state fails to the root;
       a deeper state u, entered from r on byte a, fails to goto(f, a) for the
       first f on r's failure chain that has an a-edge, else to the root. */
    int32_t *queue = (int32_t *)malloc((size_t)m->n_nodes * sizeof(int32_t));
    if (!queue) {
        oracle_ac_free(m);
        return NULL;
    }
    uint32_t qh = 0, qt = 0;
    for (int32_t c = m->nodes[0].first_child; c >= 0; c = m->nodes[c].next_sibling) {
        m->nodes[c].fail = 0;
        m->nodes[c].dict = -1;
        queue[qt++] = c;
    }
    while (qh < qt) {
        int32_t r = queue[qh++];
        for (int32_t u = m->nodes[r].first_child; u >= 0; u = m->nodes[u].next_sibling) {
            uint8_t a = m->nodes[u].byte;
            int32_t v = m->nodes[r].fail;
            while (v != 0 && oracle_goto(m, v, a) < 0) v = m->nodes[v].fail;
            int32_t g = oracle_goto(m, v, a);
            int32_t f = (g >= 0) ? g : 0;
            m->nodes[u].fail = f;
            /* output function, inherited part: output(u) = own(u) U output(f).
               Kept as a link to the next state on the chain with own keywords. */
            m->nodes[u].dict = (m->nodes[f].own_head >= 0) ? f : m->nodes[f].dict;
            queue[qt++] = u;
        }
    }
    free(queue);
    return m;
}

uint32_t oracle_ac_states(const oracle_ac *m) { return m->n_nodes; }

/* Number of states at each depth 0..max_depth (inclusive); returns the max depth. */
uint32_t oracle_ac_depth_counts(const oracle_ac *m, uint64_t *counts, uint32_t cap)
{
    uint32_t maxd = 0;
    for (uint32_t s = 0; s < m->n_nodes; ++s) {
        uint32_t d = (uint32_t)m->nodes[s].depth;
        if (d > maxd) maxd = d;
        if (d < cap) counts[d] += 1;
    }
    return maxd;
}

/*
 * The serial pass (section II): follow goto, on a missing edge follow failure,
 * and at each position emit output(state).  Writes up to cap (end, id) pairs in
 * scan order and returns the total number of occurrences.
 */
uint64_t oracle_ac_full(const oracle_ac *m, const uint8_t *text, uint64_t n,
                        uint64_t *ends, int32_t *ids, uint64_t cap)
{
    uint64_t total = 0;
    int32_t s = 0;
    for (uint64_t e = 0; e < n; ++e) {
        uint8_t a = text[e];
        while (s != 0 && oracle_goto(m, s, a) < 0) s = m->nodes[s].fail;
        int32_t t = oracle_goto(m, s, a);
        s = (t >= 0) ? t : 0;
        for (int32_t v = s; v >= 0; v = m->nodes[v].dict) {
            for (int32_t id = m->nodes[v].own_head; id >= 0; id = m->own_next[id]) {
                if (total < cap) {
                    ends[total] = e;
                    ids[total] = id;
                }
                ++total;
            }
        }
    }
    return total;
}

/*
 * Per-start longest keyword (the failureless machine's result, section II):
 * every occurrence (e, id) found by the serial pass starts at e + 1 - |id|;
 * per start keep the longest keyword, equal lengths -> the lowest id; -1 where
 * nothing starts.
 */
void oracle_ac_pfac_ids(const oracle_ac *m, const uint8_t *text, uint64_t n, int32_t *best)
{
    for (uint64_t i = 0; i < n; ++i) best[i] = -1;
    int32_t s = 0;
    for (uint64_t e = 0; e < n; ++e) {
        uint8_t a = text[e];
        while (s != 0 && oracle_goto(m, s, a) < 0) s = m->nodes[s].fail;
        int32_t t = oracle_goto(m, s, a);
        s = (t >= 0) ? t : 0;
        for (int32_t v = s; v >= 0; v = m->nodes[v].dict) {
            for (int32_t id = m->nodes[v].own_head; id >= 0; id = m->own_next[id]) {
                uint64_t len = m->klen[id];
                uint64_t start = e + 1 - len;
                int32_t cur = best[start];
                if (cur < 0 || len > m->klen[cur] || (len == m->klen[cur] && id < cur))
                    best[start] = id;
            }
        }
    }
}

/*
 * Work statistic for the failureless walk (not a result): for every start i,
 * follow goto only, from the root, until an edge is missing or the text ends;
 * count the goto evaluations.  Returns the total over all starts and the
 * largest single walk through *max_walk.
 */
uint64_t oracle_ac_walk_steps(const oracle_ac *m, const uint8_t *text, uint64_t n, uint64_t *max_walk)
{
    uint64_t total = 0, mx = 0;
    for (uint64_t i = 0; i < n; ++i) {
        int32_t s = 0;
        uint64_t steps = 0;
        for (uint64_t j = i; j < n; ++j) {
            int32_t t = oracle_goto(m, s, text[j]);
            ++steps;
            if (t < 0) break;
            s = t;
        }
        total += steps;
        if (steps > mx) mx = steps;
    }
    if (max_walk) *max_walk = mx;
    return total;
}
