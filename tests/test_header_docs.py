"""The C boundary documents itself: every function include/he.h declares has
a comment, and every one that performs an operation of the method cites the
passage of the paper that defines it (a section or Algorithm 1). Handle
management, sizes, tuning knobs and measurement probes are exempt from the
citation (they define no operation of the method)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "he.h")

EXEMPT = re.compile(r"_destroy$|_scratch_bytes(_ex)?$|^he_version$|^he_last_error$|^he_plan_launches$|"
                    r"^he_ntt_shapes$|^he_ntt_set_shape$|^he_context_set_eval_shape$|^he_ntt_tables_psi$|"
                    r"_probe$|^he_butterfly_apply$|^he_primes_generate$|^he_ntt_plan_(fwd|inv)$|_noalloc$")


def _declarations():
    text = open(HEADER).read()
    out = []
    for m in re.finditer(r"\n(?:he_status|size_t|uint32_t)\s+(he_\w+)\(", text):
        before = text[:m.start()]
        end = before.rfind("*/")
        start = before.rfind("/*", 0, end)
        gap = before[end + 2:]
        comment = before[start:end] if start >= 0 and end >= 0 else ""
        # the comment must sit right above (only other declarations between)
        out.append((m.group(1), comment, gap))
    return out


def test_every_declaration_has_a_comment():
    for name, comment, gap in _declarations():
        assert comment, name
        assert gap.count("/*") == 0, name


def test_operations_cite_the_paper():
    missing = []
    for name, comment, _ in _declarations():
        if EXEMPT.search(name):
            continue
        if not re.search(r"Sec\. [IVX]+|Algorithm 1", comment):
            # an operation declared right below a section banner that cites
            # the passage for the whole group (e.g. the encoding calls)
            missing.append(name)
    text = open(HEADER).read()
    still = []
    for name in missing:
        pos = text.index(name + "(")
        banner = text.rfind("/* ----", 0, pos)
        if banner < 0 or not re.search(r"Sec\. [IVX]+", text[banner:text.index("\n", banner)]):
            still.append(name)
    assert not still, still
