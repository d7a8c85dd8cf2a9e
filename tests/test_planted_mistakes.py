"""Planted mistakes must make a pin fail: in the oracle, the seeded input
generators, the library's multi-rank exchange, the sweep driver and the bench.

The pins in tests/test_oracle_pins.py vouch for the oracle only if a
plausible mistake in it would break one of them. Each case below copies one
oracle source (the C file or a Python module), plants one such mistake (a
dropped term, a wrong sign, index, bound or constant, a transposed operand),
and runs the pin tests against the copy in a child process. The case passes
when a pin fails there (pytest exit status 1). A mistake that crashes or
hangs the child would not count, so the mistakes are chosen to keep every
array access in bounds, and a child is given a time limit.

The seeded input generators (workloads/) get the same treatment against
tests/test_workloads_host.py: both sides of every parity test draw their
keys from them, so only their own pins can catch a mistake there.

The library's multi-rank exchange of sub-arrays (paper_2501_18977_gb300/
sharded.py) is checked the same way against tests/test_sharded_host.py, whose
gloo ranks compare it with the oracle's split filter. Its ranks are spawned
processes that import the package from disk, so each such case runs in a
shadow tree: links to the repository's directories and a package directory
whose sharded.py is the planted copy. Only mistakes that let every rank run
to its end are planted (a rank that raised would leave its peers waiting in
a collective).

The bench's host arithmetic (bench.py: max over ranks, whole-job throughput,
ratios, the traffic record's tie, the clock record, strict JSON) runs the
same way against tests/test_bench_host.py and tests/test_multirank_host.py,
and the paper-scale sweep driver (the stream-disjointness proof, the sizes,
the batch rule) against tests/test_sweeps_host.py.

Five controls run the same way with nothing planted: the unchanged C source
compiled by this harness, an unchanged oracle module and generator module
re-executed by it, and the unchanged exchange and bench in shadow trees. They
must pass every pin, which shows that a failing case fails because of its
mistake and not because of the harness.

CPU only; the children run in parallel, stopping at their first failing pin.
"""
import concurrent.futures as cf
import os
import signal
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")
PINS = os.path.join("tests", "test_oracle_pins.py")
WORKLOAD_PINS = os.path.join("tests", "test_workloads_host.py")
EXCHANGE_PINS = [os.path.join("tests", "test_sharded_host.py")]
SWEEP_PINS = os.path.join("tests", "test_sweeps_host.py")
BENCH_PINS = [os.path.join("tests", "test_bench_host.py"), os.path.join("tests", "test_multirank_host.py")]
CHILD_TIMEOUT_S = 240

# The child: point the oracle at the planted copy, then run the pins.
#   kind "c":  the C library the oracle loads is the compiled copy;
#   otherwise: the named module is re-executed from the copy before the
#              pins import anything from it.
CHILD = r"""
import importlib, sys
kind, path = sys.argv[1], sys.argv[2]
if kind == "c":
    import oracle.build as ob
    ob.build = lambda force=False: path
else:
    mod = importlib.import_module(kind)
    with open(path) as fh:
        src = fh.read()
    exec(compile(src, mod.__file__, "exec"), mod.__dict__)
import pytest
sys.exit(pytest.main(["-x", "-q", "-p", "no:cacheprovider", sys.argv[3]]))
"""

# (name, file under oracle/, [(text, replacement), ...]); every text must
# occur exactly once in its file.
C_MUTANTS = [
    # generator (splitmix64) and multipliers (Section 3.4)
    ("splitmix_shift", [("z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;",
                         "z = (z ^ (z >> 31)) * 0xbf58476d1ce4e5b9ULL;")]),
    ("splitmix_increment", [("(*state += 0x9e3779b97f4a7c15ULL)", "(*state += 0x9e3779b97f4a7c13ULL)")]),
    ("block_multiplier_even", [("a = orc_splitmix64_next(&state) | 1u;\n        } while (orc_gcd(a, M) != 1);",
                                "a = orc_splitmix64_next(&state);\n        } while (orc_gcd(a, M) != 1);")]),
    ("block_multiplier_not_coprime", [("} while (orc_gcd(a, M) != 1);", "} while (0);")]),
    ("distinct_multiplier_range", [("uint64_t range = orc_bitsel ? ORC_BLOCK_BITS - i : ORC_BLOCK_BITS;",
                                    "uint64_t range = ORC_BLOCK_BITS;")]),
    ("random_bit_multiplier_range", [("uint64_t range = orc_bitsel ? ORC_BLOCK_BITS - i : ORC_BLOCK_BITS;",
                                      "uint64_t range = orc_bitsel ? ORC_BLOCK_BITS - i : ORC_BLOCK_BITS - 1;")]),
    # linear hash (Section 3.4)
    ("hash_odd_range", [("    return y % b;\n}", "    return y % (b - 1 > 0 ? b - 1 : 1);\n}")]),
    ("hash_pow2_low_bits", [("return (y >> (64u - lg)) % b;", "return y % b;")]),
    ("hash_pow2_shift_off_by_one", [("return (y >> (64u - lg)) % b;", "return (y >> (63u - lg)) % b;")]),
    ("hash_even_fold_dropped", [("    if ((b & 1u) == 0)\n        y = y ^ (y >> 32);\n", "")]),
    # costs (Eq. 4-6)
    ("mix_new_bits_dropped", [("pow((double)j / 256.0, dk) + (double)a;", "pow((double)j / 256.0, dk);")]),
    ("mix_wrong_scale", [("pow((double)j / 256.0, dk)", "pow((double)j / 512.0, dk)")]),
    ("la_wrong_sign", [("((double)j + param * dk)", "((double)j - param * dk)")]),
    ("la_factor_k_dropped", [("return dk * pow(((double)j + param * dk)", "return pow(((double)j + param * dk)")]),
    ("exp_operands_transposed", [("pow(param, (double)j / 128.0)", "pow((double)j / 128.0, param)")]),
    ("exp_divisor_dropped", [("+ (double)a / dk;", "+ (double)a;")]),
    ("table_cost_indexed_by_j", [("orc_table[(j - a) * (k + 1) + a]", "orc_table[j * (k + 1) + a]")]),
    # bits of a block
    ("bit_selection_mode_ignored", [("if (!orc_bitsel) {", "if (1) {")]),
    ("get_bit_reversed_in_word", [("(words[8u * b + p / 64u] >> (p % 64u)) & 1u",
                                   "(words[8u * b + p / 64u] >> (63u - p % 64u)) & 1u")]),
    ("set_bit_wrong_word", [("words[8u * b + p / 64u] |= ", "words[8u * b + (p / 64u + 1u) % 8u] |= ")]),
    ("load_misses_last_bit", [("for (uint32_t p = 0; p < ORC_BLOCK_BITS; p++)\n        L += ",
                               "for (uint32_t p = 0; p + 1 < ORC_BLOCK_BITS; p++)\n        L += ")]),
    ("new_bits_negated", [("if (inF[p] && !orc_get_bit(words, b, p))\n            a++;",
                           "if (inF[p] && orc_get_bit(words, b, p))\n            a++;")]),
    # the choice (Section 3.2)
    ("skip_rule_dropped", [("        if (a[i] == 0)\n            return -1;\n", "")]),
    ("ties_to_last", [("cost < best_cost", "cost <= best_cost")]),
    ("argmax_instead_of_argmin", [("cost < best_cost", "cost > best_cost")]),
    ("cost_of_load_before_insert", [("orc_cost(kind, param, k, L + a[i], a[i])", "orc_cost(kind, param, k, L, a[i])")]),
    # batch-synchronous insertion (Section 3.1)
    ("keys_one_by_one", [("uint64_t e = (n - s) < B ? n : s + B;", "uint64_t e = s + 1;"),
                         ("for (uint64_t s = 0; s < n; s += B) {", "for (uint64_t s = 0; s < n; s += 1) {")]),
    ("last_key_dropped", [("uint64_t e = (n - s) < B ? n : s + B;", "uint64_t e = (n - s) <= B ? n - 1 : s + B;")]),
    ("skips_counted_as_inserts", [("n_skip++;", "n_ins++;")]),
    ("set_in_first_candidate", [("uint64_t b = orc_hash(a_block[(int)ch[t - s]], keys[t], M);",
                                 "uint64_t b = orc_hash(a_block[0], keys[t], M);")]),
    # query (Section 3.1)
    ("query_first_candidate_only", [("for (uint32_t i = 0; i < c && !hit; i++) {",
                                     "for (uint32_t i = 0; i < 1 && !hit; i++) {")]),
    ("query_first_hit_index", [("hit = (int)i + 1;", "hit = (int)i;")]),
    ("query_bitmap_msb_first", [("bitmap[t / 64] |= (uint64_t)1 << (t % 64);",
                                 "bitmap[t / 64] |= (uint64_t)1 << (63 - t % 64);")]),
    # load histogram (Appendix C)
    ("histogram_off_by_one", [("hist[L]++;", "hist[L > 0 ? L - 1 : 0]++;")]),
    ("histogram_total_counts_blocks", [("total += L;", "total += 1;")]),
    # distinct bit selection (Appendix B)
    ("distinct_shift_strict", [("uint32_t f = (uint32_t)orc_hash(a_bit[i], x, ORC_BLOCK_BITS - i);\n"
                                "        uint32_t pos = 0;\n        while (pos < nsorted && sorted[pos] <= f) {",
                                "uint32_t f = (uint32_t)orc_hash(a_bit[i], x, ORC_BLOCK_BITS - i);\n"
                                "        uint32_t pos = 0;\n        while (pos < nsorted && sorted[pos] < f) {")]),
    ("distinct_raw_shift_strict", [("uint32_t f = raw[i];\n        uint32_t pos = 0;\n"
                                    "        while (pos < nsorted && sorted[pos] <= f) {",
                                    "uint32_t f = raw[i];\n        uint32_t pos = 0;\n"
                                    "        while (pos < nsorted && sorted[pos] < f) {")]),
]

PY_MUTANTS = [
    # closed forms (Eq. 1, Eq. 2, Fig. 3, Appendix C)
    ("oracle.closed_forms", "bloom_fpr_k_dropped", [("math.exp(-n * k / m)", "math.exp(-n / m)")]),
    ("oracle.closed_forms", "overload_sign", [("2.0 ** (-gamma)", "2.0 ** (gamma)")]),
    ("oracle.closed_forms", "bloom_bits_times_ln2", [("n * k / math.log(2.0)", "n * k * math.log(2.0)")]),
    ("oracle.closed_forms", "load_bound_sign", [("256.0 * c ** (-1.0 / k)", "256.0 * c ** (1.0 / k)")]),
    ("oracle.closed_forms", "birthday_off_by_one", [("p *= 1.0 - i / s", "p *= 1.0 - (i + 1) / s")]),
    ("oracle.closed_forms", "blocked_bloom_bit_exponent", [("(1.0 - 1.0 / BLOCK_BITS) ** (i * k)",
                                                     "(1.0 - 1.0 / BLOCK_BITS) ** i")]),
    ("oracle.closed_forms", "state_fpr_exponent", [("(L / BLOCK_BITS) ** k", "(L / BLOCK_BITS) ** (k - 1)")]),
    ("oracle.closed_forms", "choices_fpr_linearised", [("return 1.0 - (1.0 - q) ** c", "return c * q")]),
    # learned cost: network, gradient, sampler, Adam
    ("oracle.learned", "grid_load_without_new_bits", [("(L + a) / 512.0", "L / 512.0")]),
    ("oracle.learned", "forward_bias_sign", [("return h2 @ w3 + b3", "return h2 @ w3 - b3")]),
    ("oracle.learned", "tanh_derivative_wrong", [("d1 = (d2 @ W2) * (1.0 - h1 ** 2)", "d1 = (d2 @ W2) * (1.0 - h1)")]),
    ("oracle.learned", "output_bias_gradient_dropped", [("g[5 * H + H * H] = w.sum()", "g[5 * H + H * H] = 0.0")]),
    ("oracle.learned", "second_layer_transposed", [("g[3 * H:3 * H + H * H] = (d2.T @ h1).reshape(-1)",
                                             "g[3 * H:3 * H + H * H] = (h1.T @ d2).reshape(-1)")]),
    ("oracle.learned", "uniform_bits", [("return (z >> 11) / float(1 << 53)", "return (z >> 12) / float(1 << 53)")]),
    ("oracle.learned", "policy_sign", [("e = np.exp(-(g - g.min()) / tau)", "e = np.exp((g - g.min()) / tau)")]),
    ("oracle.learned", "score_weight_tau_dropped", [("w[p] += (e[i] / z - (1.0 if i == s else 0.0)) / tau",
                                              "w[p] += (e[i] / z - (1.0 if i == s else 0.0))")]),
    ("oracle.learned", "adam_bias_correction_dropped", [("vh = m2 / (1 - b2 ** step)", "vh = m2")]),
    ("oracle.learned", "adam_betas_swapped", [("mh = m1 / (1 - b1 ** step)", "mh = m1 / (1 - b2 ** step)")]),
    # sub-arrays (Section 3.4)
    ("oracle.sharded", "h0_multiplier_even", [("a0 = out | 1", "a0 = out")]),
    ("oracle.sharded", "query_wrong_subarray", [("idx = np.flatnonzero(sh == t)",
                                          "idx = np.flatnonzero(sh == (t + 1) % self.T)")]),
    ("oracle.sharded", "layout_reversed", [("np.concatenate([s.words for s in self.subs])",
                                     "np.concatenate([s.words for s in reversed(self.subs)])")]),
    # the wrapper
    ("oracle.oracle", "bitmap_unpacked_msb_first", [('np.unpackbits(b, bitorder="little")[:n]',
                                              'np.unpackbits(b, bitorder="big")[:n]')]),
    ("oracle.oracle", "batch_argument_ignored", [("B = self.batch if batch is None else int(batch)",
                                                  "B = self.batch")]),
]


# The seeded input generators feed the oracle and the GPU path alike, so a
# mistake there survives every parity test; their own pins must catch it.
WORKLOAD_MUTANTS = [
    ("splitmix_constant", [("_M1 = np.uint64(0xBF58476D1CE4E5B9)", "_M1 = np.uint64(0xBF58476D1CE4E5B8)")]),
    ("splitmix_first_index", [("idx = np.arange(start + 1, start + n + 1, dtype=np.uint64)",
                               "idx = np.arange(start, start + n, dtype=np.uint64)")]),
    ("splitmix_at_first_index", [("idx = np.asarray(positions, dtype=np.uint64) + np.uint64(1)",
                                  "idx = np.asarray(positions, dtype=np.uint64)")]),
    ("genome_high_bits_first", [("shifts = (2 * np.arange(32, dtype=np.uint64))",
                                 "shifts = (np.uint64(62) - 2 * np.arange(32, dtype=np.uint64))")]),
    ("window_doubling_shift", [("pieces[2 * L] = (a[:m] << np.uint64(2 * L)) | a[L:L + m]",
                                "pieces[2 * L] = (a[:m] << np.uint64(L)) | a[L:L + m]")]),
    ("canonical_max", [("return np.minimum(fwd, rc)", "return np.maximum(fwd, rc)")]),
    ("complement_wrong", [("rc = _windows((3 - bases).astype(np.uint8), q, first_high=False)",
                           "rc = _windows((bases ^ 1).astype(np.uint8), q, first_high=False)")]),
    ("reverse_missing", [("rc = _windows((3 - bases).astype(np.uint8), q, first_high=False)",
                          "rc = _windows((3 - bases).astype(np.uint8), q, first_high=True)")]),
    ("disjoint_not_excluding", [("cand = cand[ex[pos] != cand]", "cand = cand")]),
    ("box_muller_sin", [("np.cos(2.0 * math.pi * u2)", "np.sin(2.0 * math.pi * u2)")]),
    ("many_filter_blocks_rounded_down", [("M = -(-bits_per_key * n // 512)", "M = bits_per_key * n // 512")]),
    ("many_filter_queries_all_members", [("return keys, np.concatenate([keys[:half], other])",
                                          "return keys, np.concatenate([keys, other])")]),
    ("serving_query_fraction", [("kind = 1 if r[j, 1] < query_frac else 0",
                                 "kind = 1 if r[j, 1] > query_frac else 0")]),
    ("serving_members_not_yet_inserted", [("n_mem) % np.uint64(have)", "n_mem) % np.uint64(have + 1)")]),
]


# The paper-scale sweep driver: the proof that inserted and negative key
# streams are disjoint, the sizes of Appendix C and the batch rule.
SWEEP_MUTANTS = [
    ("overlap_lower_bound", [("return not (d < n or d > (1 << 64) - n_neg)",
                              "return not (d < n - 1 or d > (1 << 64) - n_neg)")]),
    ("overlap_upper_bound", [("return not (d < n or d > (1 << 64) - n_neg)",
                              "return not (d < n or d >= (1 << 64) - n_neg)")]),
    ("gamma_not_inverted", [("pow(GAMMA, -1, 1 << 64)", "GAMMA")]),
    ("blocks_rounded_down", [("math.ceil(bloom_bits(n, k, rho) / 512.0)",
                              "math.floor(bloom_bits(n, k, rho) / 512.0)")]),
    ("batch_fraction", [("max(M / 64.0, 1.0)", "max(M / 32.0, 1.0)")]),
    ("batch_cap", [("max(0, min(20, ", "max(0, min(21, ")]),
    ("bloom_exponent_dropped", [("return (1.0 - math.exp(-k * n / m)) ** k", "return (1.0 - math.exp(-k * n / m))")]),
    ("poisson_mean_inverted", [("    lam = n / M\n", "    lam = M / n\n")]),
    ("bloom_bits_rho_dropped", [("return rho * n * k / LN2", "return n * k / LN2")]),
]

# The multi-rank exchange (the library's sharded.py); every rank still
# reaches its end, with wrong words or answers.
EXCHANGE_MUTANTS = [
    ("exchange_drops_first_received_key", [("    if recv.numel():\n        local_insert(recv)",
                                            "    if recv.numel() > 1:\n        local_insert(recv[1:])")]),
    ("exchange_reverses_arrival_order", [("        local_insert(recv)", "        local_insert(recv.flip(0))")]),
    ("answers_written_to_the_start", [("local_query(recv[kpos:kpos + c], answers[wpos:wpos + w])",
                                       "local_query(recv[kpos:kpos + c], answers[:w])")]),
    ("answers_of_sources_reversed", [("    for c, w in zip(rc, rw):",
                                      "    for c, w in zip(reversed(rc), reversed(rw)):")]),
]


# The measurement contract's host arithmetic (bench.py): max over ranks,
# whole-job throughput, ratios, the traffic record's tie, the clock record
# and strict JSON.
BENCH_MUTANTS = [
    ("slowest_rank_is_the_fastest", [("op=dist.ReduceOp.MAX", "op=dist.ReduceOp.MIN")]),
    ("throughput_per_rank", [("return world * keys_per_rank / (ms_per_step / 1e3) / 1e6",
                              "return keys_per_rank / (ms_per_step / 1e3) / 1e6")]),
    ("ratio_inverted", [("else round(a / b, nd)", "else round(b / a, nd)")]),
    ("traffic_launch_not_checked", [("    if d[kernel].get(\"launch\") != launch_config(tuning, kernel):\n"
                                     "        return None\n", "")]),
    ("traffic_sources_not_checked", [("    if d[kernel].get(\"sources_sha256\") != "
                                      "sources_sha256(KERNEL_SOURCES[kernel]):\n"
                                      "        return None\n", "")]),
    ("clock_median_over_all_samples", [("\"sm_mhz\": statistics.median(busy) if busy else max(sm)",
                                        "\"sm_mhz\": statistics.median(sm)")]),
    ("idle_samples_counted_busy", [("float(parts[9]) >= 50.0", "float(parts[9]) >= 0.0")]),
    ("nan_left_in_json", [("return obj if math.isfinite(obj) else None", "return obj")]),
    ("throttle_reasons_shifted", [("zip(names, parts[5:9])", "zip(names, parts[4:8])")]),
]


def _plant(src, edits):
    for old, new in edits:
        assert src.count(old) == 1, "planted text must occur exactly once: %r" % old
        src = src.replace(old, new)
    return src


def _compile_c(src, out_dir, name):
    c = os.path.join(out_dir, name + ".c")
    lib = os.path.join(out_dir, "lib" + name + ".so")
    with open(c, "w") as fh:
        fh.write(src)
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-o", lib, c, "-lm"],
                   check=True, capture_output=True)
    return lib


def _module_file(module):
    parts = module.split(".")
    base = os.path.join(ROOT, *parts)
    return os.path.join(base, "__init__.py") if os.path.isdir(base) else base + ".py"


def _run(cmd, cwd):
    """(exit status, output tail) of a child in a session of its own; on
    timeout the whole session (the child and any rank it spawned) is killed."""
    env = dict(os.environ, PYTHONDONTWRITEBYTECODE="1")
    p = subprocess.Popen(cmd, cwd=cwd, env=env, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                         text=True, start_new_session=True)
    try:
        out, _ = p.communicate(timeout=CHILD_TIMEOUT_S)
    except subprocess.TimeoutExpired:
        os.killpg(p.pid, signal.SIGKILL)
        p.communicate()
        return "timeout", ""
    return p.returncode, out[-1500:]


def _run_pins(kind, path, pins):
    """(exit status of the pins run against the planted copy, output tail)."""
    return _run([sys.executable, "-c", CHILD, kind, path, pins], ROOT)


def _shadow_tree(out_dir, name, relpath, src):
    """A tree of links to the repository in which the file at `relpath` is
    `src`: the directories on its path are real, everything else is a link."""
    top = os.path.join(out_dir, "shadow_" + name)

    def mirror(src_dir, dst_dir, rest):
        os.makedirs(dst_dir)
        for entry in os.listdir(src_dir):
            if entry.startswith(".") or entry == "__pycache__":
                continue
            if entry != rest[0]:
                os.symlink(os.path.join(src_dir, entry), os.path.join(dst_dir, entry))
            elif len(rest) == 1:
                with open(os.path.join(dst_dir, entry), "w") as fh:
                    fh.write(src)
            else:
                mirror(os.path.join(src_dir, entry), os.path.join(dst_dir, entry), rest[1:])

    mirror(ROOT, top, relpath.split("/"))
    return top


def _run_shadow_pins(top, pins):
    return _run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] + list(pins), top)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Exit status of the pins for every planted copy and every control."""
    out_dir = str(tmp_path_factory.mktemp("planted"))
    with open(os.path.join(ORACLE, "blowchoc_oracle.c")) as fh:
        c_src = fh.read()
    jobs = {"control_c": ("c", _compile_c(c_src, out_dir, "control_c"), PINS)}
    for name, edits in C_MUTANTS:
        jobs[name] = ("c", _compile_c(_plant(c_src, edits), out_dir, name), PINS)
    py = [(module, name, edits, PINS) for module, name, edits in PY_MUTANTS]
    py += [("workloads", name, edits, WORKLOAD_PINS) for name, edits in WORKLOAD_MUTANTS]
    py += [("paper_2501_18977_gb300.sweeps", name, edits, SWEEP_PINS) for name, edits in SWEEP_MUTANTS]
    py += [("oracle.closed_forms", "control_py", [], PINS), ("workloads", "control_workloads", [], WORKLOAD_PINS)]
    for module, name, edits, pins in py:
        with open(_module_file(module)) as fh:
            src = fh.read()
        path = os.path.join(out_dir, name + ".py")
        with open(path, "w") as fh:
            fh.write(_plant(src, edits))
        jobs[name] = (module, path, pins)
    shadow = [("paper_2501_18977_gb300/sharded.py", EXCHANGE_PINS, "control_exchange", [])]
    shadow += [("paper_2501_18977_gb300/sharded.py", EXCHANGE_PINS, n, e) for n, e in EXCHANGE_MUTANTS]
    shadow += [("bench.py", BENCH_PINS, "control_bench", [])]
    shadow += [("bench.py", BENCH_PINS, n, e) for n, e in BENCH_MUTANTS]
    trees = {}
    for relpath, pins, name, edits in shadow:
        with open(os.path.join(ROOT, relpath)) as fh:
            trees[name] = (_shadow_tree(out_dir, name, relpath, _plant(fh.read(), edits)), pins)
    workers = max(1, min(8, os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {name: ex.submit(_run_shadow_pins, *tree) for name, tree in trees.items()}
        futs.update({name: ex.submit(_run_pins, *job) for name, job in jobs.items()})
        return {name: f.result() for name, f in futs.items()}


@pytest.mark.parametrize("control", ["control_c", "control_py", "control_workloads", "control_exchange",
                                     "control_bench"])
def test_unplanted_copies_pass_every_pin(outcomes, control):
    rc, tail = outcomes[control]
    assert rc == 0, tail


@pytest.mark.parametrize("name", [n for n, _ in C_MUTANTS])
def test_planted_mistake_in_the_c_oracle_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 1, "planted mistake %s was not caught (exit %s):\n%s" % (name, rc, tail)


@pytest.mark.parametrize("name", [n for _, n, _ in PY_MUTANTS])
def test_planted_mistake_in_a_python_oracle_module_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 1, "planted mistake %s was not caught (exit %s):\n%s" % (name, rc, tail)


@pytest.mark.parametrize("name", [n for n, _ in WORKLOAD_MUTANTS])
def test_planted_mistake_in_the_input_generators_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 1, "planted mistake %s was not caught (exit %s):\n%s" % (name, rc, tail)


@pytest.mark.parametrize("name", [n for n, _ in EXCHANGE_MUTANTS])
def test_planted_mistake_in_the_multi_rank_exchange_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 1, "planted mistake %s was not caught (exit %s):\n%s" % (name, rc, tail)


@pytest.mark.parametrize("name", [n for n, _ in BENCH_MUTANTS])
def test_planted_mistake_in_the_bench_arithmetic_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 1, "planted mistake %s was not caught (exit %s):\n%s" % (name, rc, tail)


@pytest.mark.parametrize("name", [n for n, _ in SWEEP_MUTANTS])
def test_planted_mistake_in_the_sweep_driver_fails_a_pin(outcomes, name):
    rc, tail = outcomes[name]
    assert rc == 1, "planted mistake %s was not caught (exit %s):\n%s" % (name, rc, tail)
