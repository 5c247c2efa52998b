"""The boundary from C: include/he.h compiles as strict C99 (no C++ types,
no warnings at -Wall -Wextra -pedantic), and a C program linked against
libhe.so calls the host-only entry points (version, prime generation, host
argument checks with their messages) with no Python in between. Runs without
a GPU: nothing here enqueues device work."""
import os
import shutil
import subprocess

import pytest

import oracle
from paper_2109_14704_gb300 import he

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "he.h"

int main(void)
{
    uint64_t q[4];
    char msg[256];
    he_ntt_tables *t = NULL;
    uint64_t bad = 12289;   /* 1 mod 2N for N = 4096 but far below 2^30 */
    printf("version %u\n", (unsigned)he_version());
    if (he_primes_generate(60, 2 * 32768, 4, NULL, 0, q) != HE_OK) return 1;
    printf("primes %llu %llu %llu %llu\n", (unsigned long long)q[0], (unsigned long long)q[1],
           (unsigned long long)q[2], (unsigned long long)q[3]);
    printf("nonpow2 %d\n", (int)he_ntt_tables_create(3000, 1, q, &t));
    he_last_error(msg, sizeof msg);
    printf("message %s\n", msg);
    printf("small %d\n", (int)he_ntt_tables_create(4096, 1, &bad, &t));
    printf("unsupported %d\n", (int)he_ntt_tables_create(1u << 17, 1, q, &t));
    printf("destroy_null %d\n", (int)he_ntt_tables_destroy(NULL));
    printf("null_tables %d\n", (int)he_ntt_fwd(NULL, 4096, 1, 1, q, NULL, NULL));
    printf("handle_untouched %d\n", t == NULL);
    return 0;
}
"""


@pytest.fixture(scope="module")
def c_run(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    lib = he.library_path()
    he.load()                                   # builds libhe.so if needed
    d = tmp_path_factory.mktemp("cclient")
    src, exe = d / "client.c", d / "client"
    src.write_text(PROGRAM)
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), lib, f"-Wl,-rpath,{os.path.dirname(lib)}"],
                   check=True, capture_output=True, text=True, timeout=120)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=60).stdout
    return dict(line.split(" ", 1) for line in out.strip().splitlines())


def test_header_compiles_as_strict_c99_alone(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if not cc:
        pytest.skip("no C compiler")
    src = tmp_path / "only.c"
    src.write_text('#include "he.h"\nint he_header_only;\n')
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                    "-I", os.path.join(ROOT, "include"), str(src)], check=True, capture_output=True, timeout=60)


def test_c_program_calls_the_library(c_run):
    assert int(c_run["version"]) == he.version()
    assert [int(x) for x in c_run["primes"].split()] == oracle.find_primes(60, 2 * 32768, 4)
    assert int(c_run["nonpow2"]) == he.HE_EINVAL and "power of two" in c_run["message"]
    assert int(c_run["small"]) == he.HE_EINVAL
    assert int(c_run["unsupported"]) == he.HE_EUNSUPPORTED
    assert int(c_run["destroy_null"]) == he.HE_OK
    assert int(c_run["null_tables"]) == he.HE_EINVAL
    assert c_run["handle_untouched"] == "1"     # failed calls leave the output handle alone
