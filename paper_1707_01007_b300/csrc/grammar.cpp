// Grammar text -> normal form of Section 2 (A -> B C, A -> x) plus A -> eps.
// A terminal used inside a binary production gets a preterminal "<x>" with "<x> -> x",
// the rewrite the paper applies to its same-generation grammar in Section 4.3.
#include <cstdio>
#include <cstring>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/cfpq.h"

struct cfpq_parsed_grammar {
    std::vector<std::string> names;
    std::vector<cfpq_rule1> unary;
    std::vector<cfpq_rule2> binary;
    std::vector<int32_t> eps;
    cfpq_grammar_cnf cnf;
};

namespace {

int fail(char *err, size_t errlen, const std::string &msg) {
    if (err && errlen) snprintf(err, errlen, "%s", msg.c_str());
    return CFPQ_ERR_INVALID;
}

}  // namespace

extern "C" int cfpq_grammar_parse(const char *text, const char *const *labels, int32_t n_labels,
                                  cfpq_parsed_grammar **out, char *err, size_t errlen) {
    if (!text || !out || n_labels < 0 || (n_labels > 0 && !labels)) return fail(err, errlen, "NULL argument");
    std::map<std::string, int32_t> term;
    for (int32_t i = 0; i < n_labels; i++) {
        if (!labels[i]) return fail(err, errlen, "NULL label name");
        term.emplace(labels[i], i);
    }
    std::vector<std::vector<std::string>> rows;
    std::istringstream in(text);
    std::string line;
    while (std::getline(in, line)) {
        const size_t hash = line.find('#');
        if (hash != std::string::npos) line.resize(hash);
        std::istringstream ls(line);
        std::vector<std::string> toks;
        std::string t;
        while (ls >> t) toks.push_back(t);
        if (toks.empty()) continue;
        if (toks.size() != 2 && toks.size() != 3) return fail(err, errlen, "bad production: " + line);
        for (const auto &s : toks)
            if (s.find('<') != std::string::npos || s.find('>') != std::string::npos)
                return fail(err, errlen, "symbol may not contain '<' or '>': " + s);
        rows.push_back(toks);
    }
    auto pg = new cfpq_parsed_grammar();
    std::map<std::string, int32_t> nt;
    for (const auto &r : rows) {
        if (r[0] == "eps") { delete pg; return fail(err, errlen, "'eps' cannot be a left-hand side"); }
        if (!nt.count(r[0])) {
            nt[r[0]] = (int32_t)pg->names.size();
            pg->names.push_back(r[0]);
        }
    }
    std::vector<std::string> pre_order;
    std::map<std::string, int32_t> pre;
    struct Pending { int32_t a; std::string b, c; };
    std::vector<Pending> pending;
    for (const auto &r : rows) {
        const int32_t a = nt[r[0]];
        if (r.size() == 2) {
            if (r[1] == "eps") {
                pg->eps.push_back(a);
            } else if (nt.count(r[1])) {
                delete pg;
                return fail(err, errlen, "chain production " + r[0] + " -> " + r[1] + " is not in normal form");
            } else if (term.count(r[1])) {
                pg->unary.push_back({a, term[r[1]]});
            } else {
                delete pg;
                return fail(err, errlen, "unknown terminal " + r[1]);
            }
        } else {
            for (int k = 1; k <= 2; k++) {
                const std::string &s = r[k];
                if (s == "eps") { delete pg; return fail(err, errlen, "eps inside a binary production"); }
                if (nt.count(s)) continue;
                if (!term.count(s)) { delete pg; return fail(err, errlen, "unknown terminal " + s); }
                if (!pre.count(s)) { pre[s] = -1; pre_order.push_back(s); }
            }
            pending.push_back({a, r[1], r[2]});
        }
    }
    for (const auto &s : pre_order) {
        pre[s] = (int32_t)pg->names.size();
        pg->names.push_back("<" + s + ">");
        pg->unary.push_back({pre[s], term[s]});
    }
    for (const auto &p : pending) {
        const int32_t b = nt.count(p.b) ? nt[p.b] : pre[p.b];
        const int32_t c = nt.count(p.c) ? nt[p.c] : pre[p.c];
        pg->binary.push_back({p.a, b, c});
    }
    if ((int)pg->names.size() > CFPQ_MAX_NONTERM) {
        delete pg;
        return fail(err, errlen, "too many non-terminals");
    }
    pg->cnf.n_nonterm = (int32_t)pg->names.size();
    pg->cnf.n_term = n_labels;
    pg->cnf.unary = pg->unary.data();
    pg->cnf.n_unary = (int32_t)pg->unary.size();
    pg->cnf.binary = pg->binary.data();
    pg->cnf.n_binary = (int32_t)pg->binary.size();
    pg->cnf.eps_lhs = pg->eps.data();
    pg->cnf.n_eps = (int32_t)pg->eps.size();
    *out = pg;
    return CFPQ_OK;
}

extern "C" const cfpq_grammar_cnf *cfpq_grammar_cnf_of(const cfpq_parsed_grammar *pg) {
    return pg ? &pg->cnf : nullptr;
}

extern "C" const char *cfpq_grammar_name(const cfpq_parsed_grammar *pg, int32_t id) {
    if (!pg || id < 0 || id >= (int32_t)pg->names.size()) return nullptr;
    return pg->names[id].c_str();
}

extern "C" void cfpq_grammar_free(cfpq_parsed_grammar *pg) { delete pg; }
