"""Static checks of the device sources (no GPU): every wait on an mbarrier
is bounded by a deadline, and no kernel traps.  A kernel that spins on a
barrier without a deadline, or stops itself with a trap, can leave a GPU
unusable for whoever uses it next; the watchdog design (a deadline on every
wait, an error status for the host, every role leaving its loop) depends on
each spin having its own exit."""
import os
import re

CSRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2310_20347_gb300", "csrc")
DEVICE = [f for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cuh"))]


def _code(name):
    text = open(os.path.join(CSRC, name)).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    return re.sub(r"//[^\n]*", " ", text)


def _loop_body(code, start):
    """The text of the while loop starting at `start`: its condition and the
    statement or braced block after it."""
    i = code.index("(", start)
    depth = 0
    while True:
        depth += {"(": 1, ")": -1}.get(code[i], 0)
        i += 1
        if depth == 0:
            break
    rest = code[i:].lstrip()
    j = len(code) - len(rest)
    if rest.startswith("{"):
        depth = 0
        k = j
        while True:
            depth += {"{": 1, "}": -1}.get(code[k], 0)
            k += 1
            if depth == 0:
                return code[start:k]
    return code[start:code.index(";", j) + 1]


def _parenthesised(code, i):
    """The text between the parenthesis at code[i] and its match."""
    depth, j = 0, i
    while True:
        depth += {"(": 1, ")": -1}.get(code[j], 0)
        j += 1
        if depth == 0:
            return code[i + 1:j - 1]


def _top_level_commas(args):
    depth, n = 0, 0
    for ch in args:
        depth += {"(": 1, ")": -1, "<": 0, ">": 0}.get(ch, 0)
        n += ch == "," and depth == 0
    return n


def test_every_barrier_spin_has_a_deadline():
    spins = 0
    for name in DEVICE:
        code = _code(name)
        for m in re.finditer(r"\bwhile\s*\(", code):
            body = _loop_body(code, m.start())
            if "try_wait" not in body:
                continue
            spins += 1
            assert "globaltimer_ns()" in body and "timeout" in body, f"{name}: unbounded spin: {body[:160]}"
    assert spins >= 3   # the generic bounded wait and the drain loops


def test_waits_go_through_the_watchdog():
    # outside ptx.cuh (which defines them) the raw try-wait primitives appear
    # only inside bounded loops, checked above; every other wait is
    # wait_parity(bar, parity, watchdog, code)
    for name in DEVICE:
        if name == "ptx.cuh":
            continue
        code = _code(name)
        for m in re.finditer(r"\bwait_parity\s*(<[^>]*>)?\s*\(", code):
            args = _parenthesised(code, m.end() - 1)
            assert _top_level_commas(args) == 3, f"{name}: wait_parity without a watchdog: {args[:120]}"


def test_no_kernel_traps():
    for name in DEVICE:
        code = _code(name)
        assert "__trap" not in code, name
        assert not re.search(r"\btrap\s*;", code), name
        assert not re.search(r"\bassert\s*\(", code.replace("static_assert", "")), name
