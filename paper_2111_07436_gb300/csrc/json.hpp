// Minimal JSON reader for mechanism descriptions (objects, arrays, strings,
// numbers, true/false/null).  Object key order is preserved, because the
// declaration order of species and processes defines the state layout.
#pragma once
#include <cstdlib>
#include <memory>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

namespace campjson {

struct Value {
    enum Kind { Null, Bool, Number, String, Array, Object } kind = Null;
    bool b = false;
    double num = 0.0;
    std::string str;
    std::vector<Value> arr;
    std::vector<std::pair<std::string, Value>> obj;

    const Value *find(const std::string &k) const {
        for (auto &kv : obj)
            if (kv.first == k) return &kv.second;
        return nullptr;
    }
    const Value &at(const std::string &k) const {
        const Value *v = find(k);
        if (!v) throw std::runtime_error("missing key '" + k + "'");
        return *v;
    }
    double number(const std::string &k) const {
        const Value &v = at(k);
        if (v.kind != Number) throw std::runtime_error("key '" + k + "' is not a number");
        return v.num;
    }
    double number_or(const std::string &k, double d) const {
        const Value *v = find(k);
        if (!v) return d;
        if (v->kind != Number) throw std::runtime_error("key '" + k + "' is not a number");
        return v->num;
    }
    const std::string &string(const std::string &k) const {
        const Value &v = at(k);
        if (v.kind != String) throw std::runtime_error("key '" + k + "' is not a string");
        return v.str;
    }
};

class Parser {
  public:
    Parser(const char *s, size_t n) : p_(s), end_(s + n) {}
    Value parse() {
        Value v = value(0);
        ws();
        if (p_ != end_) fail("trailing characters");
        return v;
    }

  private:
    const char *p_, *end_;
    [[noreturn]] void fail(const char *what) {
        throw std::runtime_error(std::string("JSON: ") + what);
    }
    void ws() {
        while (p_ < end_ && (*p_ == ' ' || *p_ == '\n' || *p_ == '\t' || *p_ == '\r')) ++p_;
    }
    bool lit(const char *s) {
        size_t n = 0;
        while (s[n]) ++n;
        if ((size_t)(end_ - p_) >= n && std::string(p_, n) == s) {
            p_ += n;
            return true;
        }
        return false;
    }
    Value value(int depth) {
        if (depth > 64) fail("nesting too deep");
        ws();
        if (p_ >= end_) fail("unexpected end");
        Value v;
        char c = *p_;
        if (c == '{') {
            v.kind = Value::Object;
            ++p_;
            ws();
            if (p_ < end_ && *p_ == '}') { ++p_; return v; }
            for (;;) {
                ws();
                if (p_ >= end_ || *p_ != '"') fail("expected key");
                std::string k = string();
                ws();
                if (p_ >= end_ || *p_ != ':') fail("expected ':'");
                ++p_;
                v.obj.emplace_back(std::move(k), value(depth + 1));
                ws();
                if (p_ < end_ && *p_ == ',') { ++p_; continue; }
                if (p_ < end_ && *p_ == '}') { ++p_; break; }
                fail("expected ',' or '}'");
            }
        } else if (c == '[') {
            v.kind = Value::Array;
            ++p_;
            ws();
            if (p_ < end_ && *p_ == ']') { ++p_; return v; }
            for (;;) {
                v.arr.push_back(value(depth + 1));
                ws();
                if (p_ < end_ && *p_ == ',') { ++p_; continue; }
                if (p_ < end_ && *p_ == ']') { ++p_; break; }
                fail("expected ',' or ']'");
            }
        } else if (c == '"') {
            v.kind = Value::String;
            v.str = string();
        } else if (lit("true")) {
            v.kind = Value::Bool;
            v.b = true;
        } else if (lit("false")) {
            v.kind = Value::Bool;
        } else if (lit("null")) {
            v.kind = Value::Null;
        } else {
            v.kind = Value::Number;
            const char *s = p_;
            while (p_ < end_ && (std::isdigit((unsigned char)*p_) || *p_ == '-' || *p_ == '+' ||
                                 *p_ == '.' || *p_ == 'e' || *p_ == 'E'))
                ++p_;
            if (p_ == s) fail("unexpected character");
            std::string tok(s, p_);
            char *e = nullptr;
            v.num = std::strtod(tok.c_str(), &e);
            if (!e || *e) fail("bad number");
        }
        return v;
    }
    std::string string() {
        ++p_;  // opening quote
        std::string out;
        while (p_ < end_ && *p_ != '"') {
            if (*p_ == '\\') {
                ++p_;
                if (p_ >= end_) fail("bad escape");
                char e = *p_++;
                switch (e) {
                case '"': out += '"'; break;
                case '\\': out += '\\'; break;
                case '/': out += '/'; break;
                case 'n': out += '\n'; break;
                case 't': out += '\t'; break;
                case 'r': out += '\r'; break;
                case 'b': out += '\b'; break;
                case 'f': out += '\f'; break;
                case 'u': {
                    if (end_ - p_ < 4) fail("bad \\u escape");
                    unsigned cp = (unsigned)std::strtoul(std::string(p_, 4).c_str(), nullptr, 16);
                    p_ += 4;
                    if (cp < 0x80) out += (char)cp;
                    else if (cp < 0x800) { out += (char)(0xC0 | (cp >> 6)); out += (char)(0x80 | (cp & 0x3F)); }
                    else { out += (char)(0xE0 | (cp >> 12)); out += (char)(0x80 | ((cp >> 6) & 0x3F)); out += (char)(0x80 | (cp & 0x3F)); }
                    break;
                }
                default: fail("bad escape");
                }
            } else {
                out += *p_++;
            }
        }
        if (p_ >= end_) fail("unterminated string");
        ++p_;
        return out;
    }
};

inline Value parse(const char *s, size_t n) { return Parser(s, n).parse(); }

}  // namespace campjson
