"""Benchmark of the tDPD + RBC step on GB300.

One bench step is one time step of the whole hot path (binning and sort,
membrane forces, pair force + flux, velocity-Verlet update). The default
workload is the batched ensemble the metric is quoted on: 512 independent
replicas of uneven size (cubic periodic boxes of side 8..16 at density 3,
0..4 membranes of 500 vertices each, log-uniform permeability, uniform body
force; 3.50 M particles) advanced together in one graph-captured step, and
compared with the same replicas advanced one after another on the same GPU.
The metric is particle-steps/s.

Native arm (default): libtdpd.so through its C ABI. Each timed step is one
replay of the captured step graph; an L2 flush (a write larger than the
129 MB L2) separates the timed steps. An equal number of replays of the
instrumented graph (CUDA event nodes around each kernel, on the kernels'
stream) follows inside the timed region and gives the per-kernel durations.
Reference arm (--impl reference): the FP64 CPU oracle on the host cores.

N > 1 (torchrun): replicas only -- every rank advances its own copy of the
workload (different seed); value sums the particle-steps of all ranks over
the slowest rank's time.
"""

from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = 'tDPD particle-steps/s on 1 GB300 (% HBM roofline); batched vs plain at tol'
UNIT = 'particle-steps/s'
# DRAM bytes (read + write) of one pair step (k_pair, plus k_pair_finish in
# half-shell mode) from an ncu capture of the current kernel build (summaries
# under profiles/), keyed by workload, skin, stencil width, lane count, pair
# mode and replica count (0: not an ensemble). The ensemble's figure is the
# mean of two steps captured on its first 128 replicas (841,109 particles),
# scaled by particles to all 512 (3,496,044). The capture is cold-cache and
# the bench step follows an L2 flush, so the two see the same misses. A
# workload without an entry reports traffic null.
PAIR_TRAFFIC = {
    ('ensemble', 0.2, 2, 1, 2, 512): 2.393e9,
}


def _ns10(d):
    d['kappa'][...] = np.linspace(0.5, 2.0, int(d['n_species']), dtype=np.float32)
    return d


WORKLOADS = {
    'single_rbc': ('single RBC (500-vertex biconcave, WLC-POW, kb=20kT, area/volume constraints, '
                   'membrane viscosity) in tDPD solvent, 20^3 periodic box, rho=3, 24,500 particles, '
                   '1 species, permeability 0.1, dt=0.005', lambda seed: [W.single_rbc(seed=1002 + seed)]),
    'fluid_4k': ('plain tDPD fluid, 10^3 periodic box, rho=4, 4000 particles, 1 species',
                 lambda seed: [W.fluid_box(seed=1001 + seed)]),
    'fluid_786k': ('plain tDPD fluid, 64^3 periodic box, rho=3, 786,432 particles, 1 species '
                   '(state larger than L2; profiling case)',
                   lambda seed: [W.fluid_box(L=64.0, rho=3.0, seed=2001 + seed)]),
    'fluid_786k_ns10': ('plain tDPD fluid, 64^3 periodic box, rho=3, 786,432 particles, 10 species '
                        '(kappa 0.5..2), the multi-species case of the paper\'s fluid benchmark',
                        lambda seed: [_ns10(W.fluid_box(L=64.0, rho=3.0, n_species=10, seed=2002 + seed))]),
    'channel': ('RBC suspension: 64x32x32 channel with frozen-particle walls, 40 RBCs, 2 species, '
                'reaction k=0.01, body force 0.05, dt=0.005',
                lambda seed: [W.rbc_channel(seed=1003 + seed)]),
    'ensemble': ('512 independent replicas (cubic boxes 8..16 at rho=3, 0..4 RBCs, log-uniform '
                 'permeability, body force) batched in one graph-captured step',
                 lambda seed, n_rep=512: W.replica_ensemble(n_rep=n_rep, seed=1004 + seed)),
}


def peaks():
    try:
        with open(os.path.join(ROOT, 'MEASURED_PEAKS.json')) as f:
            p = json.load(f)
        return float(p['hbm_gbs']), 'measured'
    except Exception:
        return 6800.0, 'fallback'


def sm_max_mhz():
    try:
        with open(os.path.join(ROOT, 'MEASURED_PEAKS.json')) as f:
            return float(json.load(f)['sm_max_mhz'])
    except Exception:
        return 2070.0


def dist_env():
    rank = int(os.environ.get('RANK', '0'))
    world = int(os.environ.get('WORLD_SIZE', '1'))
    local = int(os.environ.get('LOCAL_RANK', '0'))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ('index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,'
         'clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,'
         'clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap')

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile('w+', suffix='.csv', delete=False)
        self.p = None

    def __enter__(self):
        try:
            self.p = subprocess.Popen(['nvidia-smi', '-i', str(self.index), '--query-gpu=' + self.Q,
                                       '--format=csv,noheader,nounits', '-lms', '20'],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.p:
            self.p.terminate()
            try:
                self.p.wait(timeout=5)
            except Exception:
                self.p.kill()

    def summary(self):
        try:
            rows = [l.split(',') for l in open(self.f.name).read().strip().splitlines() if l.strip()]
        except Exception:
            rows = []
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ['hw_slowdown', 'hw_thermal_slowdown', 'sw_thermal_slowdown', 'sw_power_cap']
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for k, nm in enumerate(names):
                    if r[5 + k].strip().lower() == 'active':
                        reasons.add(nm)
            except Exception:
                pass
        if not sm:
            return {'sm_mhz': None, 'sm_max_mhz': None, 'reasons': ['unsampled']}
        return {'sm_mhz': statistics.median(sm), 'sm_max_mhz': max(mx), 'reasons': sorted(reasons),
                'samples': len(sm)}


def combine_ranks(total_ms, n_particles, steps, world, device):
    """Whole-job throughput of independent replicas: particle-steps summed over
    the ranks, divided by the slowest rank's time. Returns (max ms, value)."""
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
        c = torch.tensor([float(n_particles)], device=device, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
        total_ms, n_particles = float(t.item()), float(c.item())
    return total_ms, n_particles * steps / (total_ms * 1e-3)


def oracle_rate(desc, seconds=12.0, max_steps=400):
    """FP64 oracle (cell-list mode, OpenMP on all host cores) on the workload:
    steps until ~seconds of CPU work; returns particle-steps/s, steps, cores."""
    import oracle
    o = oracle.Oracle(desc, mode=1)
    n = W.n_mobile(desc)
    t0 = time.perf_counter()
    steps = 0
    while steps < max_steps:
        o.run(1)
        steps += 1
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return n * steps / dt, steps, oracle.num_threads()


def make_descs(args, rank):
    """The workload's replica descriptions with the command line's options."""
    gen = WORKLOADS[args.workload][1]
    descs = gen(rank, args.replicas) if args.workload == 'ensemble' else gen(rank)
    for d in descs:
        d['cells_per_cutoff'] = args.cells_per_cutoff
        d['skin'] = args.skin
        d['lanes'] = args.lanes or None
        if args.lagged_av and d.get('membrane'):
            d['membrane']['lagged_av'] = 1
        if args.random_flux > 0:
            d['random_flux'] = dict(m_s=args.random_flux, rho=3.0)
    return descs


def common_config(args, descs, world):
    """The workload keys of the JSON line (identical in both arms)."""
    desc = WORKLOADS[args.workload][0]
    if args.workload == 'ensemble' and args.replicas != 512:
        desc = desc.replace('512 independent', '%d independent' % args.replicas)
    return {'workload': desc, 'name': args.workload, 'replicas': len(descs),
            'particles': sum(W.n_mobile(d) for d in descs),
            'l2': 'flushed between timed steps (256 MB write)',
            'area_volume': 'previous step (lagged)' if args.lagged_av else 'current step',
            'random_flux': {'m_s': args.random_flux, 'rho': 3.0} if args.random_flux > 0 else 'off',
            'parallelism': 'replicas only' if world > 1 else 'single GPU'}


# particle-steps of oracle work the reference arm may spend (about two
# minutes on 16 host cores at the oracle's 1.5 M particle-steps/s)
REFERENCE_BUDGET = 1.8e8


def run_reference(args):
    """The FP64 oracle (cell list, OpenMP on every host core) on the same
    workload: W untimed and K timed steps over a bounded sample (the
    replicas in order while (K + W + 1) x their particles stay within the
    budget; the default 20 + 5 steps take the whole 512-replica ensemble)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    descs = make_descs(args, 0)
    sample, work = [], 0.0
    for d in descs:
        w = W.n_particles(d) * (args.steps + args.warmup + 1)
        if sample and work + w > REFERENCE_BUDGET:
            break
        sample.append(d)
        work += w
    n = sum(W.n_mobile(d) for d in sample)
    orcs = [oracle.Oracle(d, mode=1) for d in sample]
    for _ in range(args.warmup):
        for o in orcs:
            o.run(1)
    total = 0.0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        for o in orcs:
            o.run(1)
        total += time.perf_counter() - t0
    value = n * args.steps / total
    cores = oracle.num_threads()
    what = ('the whole workload' if len(sample) == len(descs) else
            'the first %d of %d replicas' % (len(sample), len(descs)))
    line = {
        'impl': 'reference', 'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': world,
        'steps': args.steps, 'warmup': args.warmup, 'ms_per_step': 1e3 * total / args.steps,
        'higher_is_better': True, 'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f64',
        'data': 'synthetic', 'config': common_config(args, descs, world),
        'cpu_baseline': {'value': value, 'unit': UNIT, 'cores': cores, 'kind': 'oracle',
                         'sample': '%s (%d mobile particles), %d oracle steps each (FP64 cell list, OpenMP)' % (
                             what, n, args.steps)},
        'e2e': {'value': value, 'unit': UNIT, 'h2d_bytes_per_step': 0, 'd2h_bytes_per_step': 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_native(args):
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group('nccl', device_id=torch.device('cuda', local))
    import paper_1611_06163_gb300 as pkg
    pkg.build()
    from paper_1611_06163_gb300 import binding as bd

    descs = make_descs(args, rank)
    n = sum(W.n_mobile(d) for d in descs)
    stream = torch.cuda.Stream()
    if len(descs) == 1:
        parts = []
        h = bd.create_from(descs[0], stream_ptr=stream.cuda_stream)
    else:
        parts = [bd.create_from(d) for d in descs]
        h = bd.tdpd_batch_create(parts)
        bd.tdpd_set_stream(h, stream.cuda_stream)
        if args.skin is not None:
            bd.tdpd_set_skin(h, args.skin)
        if args.lanes:
            bd.tdpd_set_lanes(h, args.lanes)
    if args.pair_mode:
        bd.tdpd_set_pair_mode(h, args.pair_mode)
    if args.sort_mode:
        bd.tdpd_set_sort_mode(h, args.sort_mode)
    bd.tdpd_commit(h)
    nk = bd.tdpd_launches_per_step(h)
    # timed entries: one per launch, except that the half shell's pair entry
    # spans its two launches (k_pair and k_pair_finish)
    names = []
    while bd.tdpd_kernel_name(h, len(names)) is not None:
        names.append(bd.tdpd_kernel_name(h, len(names)))
    pair_mode = bd.tdpd_pair_mode(h)
    sort_mode, sort_ms = bd.tdpd_sort_mode(h)
    shape_skin, shape_m, shape_ms = bd.tdpd_list_shape(h)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device='cuda')

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()

    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            flush.fill_(1.0)
            bd.tdpd_step_timed(h)
    bd.tdpd_sync(h)

    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    kms = []
    rebuilds0 = sum(bd.tdpd_list_rebuilds(h, r) for r in range(len(descs)))
    barrier()
    with Clocks(local) as clk:
        t_wall = time.perf_counter()
        with torch.cuda.stream(stream):
            # production graph replays (one step each), L2 flushed in between
            for k in range(args.steps):
                flush.fill_(float(k))            # evict the previous step's state from L2
                ev[k][0].record(stream)
                bd.tdpd_step(h, 1)
                ev[k][1].record(stream)
            # the same number of replays of the instrumented graph (event
            # nodes around each kernel, on the kernels' stream) for the
            # per-kernel durations; event nodes serialise the kernels, so
            # these replays are not part of the step time
            for k in range(args.steps):
                flush.fill_(float(k))
                kms.append(bd.tdpd_step_timed(h))
        barrier()
        t_wall = time.perf_counter() - t_wall
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    bd.tdpd_sync(h)
    # list rebuilds per replica-step over the timed and the instrumented replays
    rebuild_rate = (sum(bd.tdpd_list_rebuilds(h, r) for r in range(len(descs))) - rebuilds0) / (
        2.0 * args.steps * len(descs))
    total_ms, value = combine_ranks(total_ms, n, args.steps, world, 'cuda')

    # dominant kernel: the pair force + flux + update
    K = np.array(kms)
    mean_k = K.mean(axis=0)
    ipair = names.index('pair')
    pair_ms = float(mean_k[ipair])
    # The pair kernel is bound by instruction issue, not by memory: its roof
    # is the lane-operation rate (SMs x 128 FP32 lanes x the maximum SM
    # clock; derived, not measured). Algorithmic operations per particle-step,
    # counted from the equations: every ordered pair inside the flux cut-off
    # costs 20 + 4 (ns - 1) lane operations, every pair inside the force
    # cut-off another 110 (TEA-8 draw, Box-Muller, Eq. 3); pair counts are the
    # workload's mean density times the cut-off spheres. With neighbour lists
    # the lists the kernel builds on rebuild steps add one distance test (9
    # operations) per list entry at the measured rebuild rate.
    # Bytes: the compulsory pair bytes (read r, v~ 16 B each and C~ 4 B per
    # species; write F 16 B and Q 4 B per species: 48 + 8 ns) give the HBM
    # fraction; what the implementation moves besides -- the fused corrector
    # (read v, F, C, Q of the last step, write v, C: 48 + 12 ns), the list
    # entries (4 B per partner within rcut + skin, 16 B build position) and
    # their rebuilds, or in cell mode the next binning (8 B) -- is listed
    # separately.
    ns = int(descs[0]['n_species'])
    n_all = sum(W.n_particles(d) for d in descs)
    vol = sum(float(np.prod(d['L'])) for d in descs)
    rho = n_all / vol
    d0 = descs[0]
    n_flux = rho * 4.0 / 3.0 * math.pi * float(d0['rcc']) ** 3
    n_force = rho * 4.0 / 3.0 * math.pi * float(d0['rc']) ** 3
    ops_pp = n_flux * (20 + 4 * (ns - 1)) + n_force * 110
    if args.random_flux > 0:
        # one TEA-8 draw + Box-Muller per two species, and ~8 operations per
        # species, for every pair inside the flux cut-off
        ops_pp += n_flux * (110 * ((ns + 1) // 2) + 8 * ns)
    skin = shape_skin
    rcut = max(float(d0['rc']), float(d0['rcc']))
    n_list = rho * 4.0 / 3.0 * math.pi * (rcut + skin) ** 3 if skin > 0 else 0.0
    compulsory_pp = 48 + 8 * ns
    impl = {'corrector': 48 + 12 * ns}
    if skin > 0:
        # half shell: each pair listed once (half the entries), and the
        # finishing pass reads and clears the fixed-point accumulators (32 +
        # 8 ns B) and reads back the own sums (16 + 4 ns B) written before
        n_entries = n_list / 2 if pair_mode == 2 else n_list
        ops_pp += rebuild_rate * 9 * n_entries
        impl['lists'] = 4 * n_entries + 16
        impl['list_rebuilds'] = rebuild_rate * (4 * n_entries + 16)
        if pair_mode == 2:
            impl['half_shell_sums'] = 2 * (32 + 8 * ns) + 2 * (16 + 4 * ns)
    else:
        impl['next_binning'] = 8
    hbm, src = peaks()
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sm * 128 * sm_max_mhz() * 1e6 / 1e12
    alu = ops_pp * n_all / (pair_ms * 1e-3) / 1e12
    gbs = compulsory_pp * n_all / (pair_ms * 1e-3) / 1e9
    lanes_now = bd.tdpd_lanes(h)
    traffic = None
    key = (args.workload, round(skin, 3), shape_m, lanes_now, pair_mode,
           args.replicas if args.workload == 'ensemble' else 0)
    if not args.random_flux and not args.cells_per_cutoff and key in PAIR_TRAFFIC:
        traffic = PAIR_TRAFFIC[key]
    roof = {'bound': 'alu', 'achieved': alu, 'peak': alu_peak, 'unit': 'Tops/s', 'frac': alu / alu_peak,
            'traffic': traffic, 'traffic_unit': 'bytes per pair step (ncu DRAM read + write)',
            'peak_source': 'derived: %d SMs (this device) x 128 FP32 lanes x %.0f MHz (measured max clock)' % (
                n_sm, sm_max_mhz()),
            'kernel': 'k_pair' + (' + k_pair_finish' if pair_mode == 2 else ''),
            'ops_per_particle': ops_pp, 'particles_per_launch': n_all,
            'hbm': {'achieved': gbs, 'peak': hbm, 'unit': 'GB/s', 'frac': gbs / hbm, 'peak_source': src,
                    'bytes_per_particle': compulsory_pp,
                    'implementation_bytes_per_particle': impl,
                    'all_bytes_frac': sum(impl.values()) * n_all / (pair_ms * 1e-3) / 1e9 / hbm + gbs / hbm},
            'kernel_ms': {nm: float(m) for nm, m in zip(names, mean_k)}}

    # end to end through the public API: every replica's state in from pinned
    # host memory (tdpd_set_states: one upload for the whole batch), one step,
    # the first replica's observables out
    st_all = [bd.tdpd_read_state(h, r, ns) for r in range(len(descs))]
    pos, vel, conc = (np.concatenate([x[k] for x in st_all]) for k in range(3))
    hp = torch.from_numpy(pos).pin_memory()
    hv = torch.from_numpy(vel).pin_memory()
    hc = torch.from_numpy(conc).pin_memory()
    e2e_steps = max(3, min(args.steps, 50))
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        bd.tdpd_set_states(h, hp.numpy(), hv.numpy(), hc.numpy())
        bd.tdpd_step(h, 1)
        bd.tdpd_read_observables(h, 0)
    barrier()
    e2e_s = time.perf_counter() - t0
    e2e = {'value': world * n * e2e_steps / e2e_s, 'unit': UNIT,
           'h2d_bytes_per_step': int(pos.nbytes + vel.nbytes + conc.nbytes),
           'd2h_bytes_per_step': 8 * (6 + 2 * bd.MAX_SPECIES),   # the binary64 totals tdpd_read_observables copies
           'path': 'tdpd_set_states (pinned host, every replica) + tdpd_step(1) + tdpd_read_observables'}

    # batched vs plain: the same replicas advanced one after another, each by
    # its own handle, against the batch (both back to back on one stream)
    lanes = bd.tdpd_lanes(h)
    compare = None
    if args.compare_sequential and len(descs) > 1:
        K = max(1, args.compare_steps)
        singles = []
        for d in descs:
            hs_ = bd.create_from(d, stream_ptr=stream.cuda_stream)
            bd.tdpd_commit(hs_)
            singles.append(hs_)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            bd.tdpd_step(h, K)                         # warm
            for hs_ in singles:
                bd.tdpd_step(hs_, K)
            torch.cuda.synchronize()
            e0.record(stream)
            bd.tdpd_step(h, K)
            e1.record(stream)
            torch.cuda.synchronize()
            t_batch = e0.elapsed_time(e1)
            e0.record(stream)
            for hs_ in singles:
                bd.tdpd_step(hs_, K)
            e1.record(stream)
            torch.cuda.synchronize()
            t_seq = e0.elapsed_time(e1)
        for hs_ in singles:
            bd.tdpd_destroy(hs_)
        compare = {'steps': K, 'replicas': len(descs),
                   'batched': n * K / (t_batch * 1e-3), 'sequential': n * K / (t_seq * 1e-3),
                   'ratio': t_seq / t_batch, 'unit': UNIT,
                   'accuracy': 'the same kernels; at equal lane counts a replica in the batch gives the same '
                               'bits as alone (tested); here every handle uses the lane count it timed'}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sample = descs[:8]
        rate, steps, cores = 0.0, 0, 0
        for d in sample:
            r_, s_, cores = oracle_rate(d, seconds=args.cpu_seconds / len(sample))
            rate += 1.0 / r_ * W.n_mobile(d)
            steps += s_
        rate = sum(W.n_mobile(d) for d in sample) / rate
        cpu = {'value': rate, 'unit': UNIT, 'cores': cores, 'kind': 'oracle',
               'sample': '%s, %d FP64 oracle steps in all, about %.0f s per replica (cell list, OpenMP); '
                         'value = their particles over the summed per-replica step times' % (
                   'full workload' if len(sample) == len(descs) else
                   'first %d of %d replicas' % (len(sample), len(descs)), steps, args.cpu_seconds / len(sample))}
    bd.tdpd_destroy(h)
    for hp_ in parts:
        bd.tdpd_destroy(hp_)
    if rank == 0:
        line = {
            'metric': METRIC, 'value': value, 'unit': UNIT, 'n_gpus': world, 'steps': args.steps,
            'warmup': args.warmup, 'ms_per_step': total_ms / args.steps, 'higher_is_better': True,
            'scaling': 'weak', 'vs_baseline': None, 'dtype': 'f32', 'data': 'synthetic',
            'config': common_config(args, descs, world),
            'tuning': {'lanes_per_particle': lanes,
                       'pair_mode': {1: 'full shell', 2: 'half shell (fixed-point partner sums)'}.get(pair_mode),
                       'neighbour_list': ({'skin': skin, 'rebuilds_per_replica_step': rebuild_rate} if skin > 0
                                          else 'off (cell stencil every step)'),
                       'cells_per_cutoff': shape_m,
                       'shape': ('timed at commit: ms per 16 steps for skins 0.2, 0.15, 0.25, 0.3, 0.4 at m = 2'
                                 '%s' % (', then at m = 3' if len(shape_ms) > 5 else '')) if len(shape_ms) else
                                'not timed (pinned)',
                       'shape_ms': [round(float(x), 4) for x in shape_ms],
                       'sort': ({1: 'kernel chain', 2: 'one thread-block cluster'}.get(sort_mode) if skin > 0
                                else 'kernel chain (cell mode)'),
                       'sort_ms': ([round(float(x), 4) for x in sort_ms] if (sort_ms > 0).all() else
                                   'not timed')},
            'roofline': roof,
            'cpu_baseline': cpu,
            'e2e': e2e,
            'gpu_launches': 2 * nk * args.steps,
            'clocks': clk.summary(),
            'batched_vs_plain': compare,
            'wall_s': t_wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument('--gpus', type=int, default=1)
    ap.add_argument('--steps', type=int, default=200)
    ap.add_argument('--warmup', type=int, default=10)
    ap.add_argument('--impl', default='native', choices=['native', 'reference'])
    ap.add_argument('--cpu-seconds', type=float, default=12.0)
    ap.add_argument('--no-cpu-baseline', action='store_true')
    ap.add_argument('--workload', default='ensemble', choices=sorted(WORKLOADS))
    ap.add_argument('--replicas', type=int, default=512, help='ensemble only: number of replicas')
    ap.add_argument('--no-compare-sequential', dest='compare_sequential', action='store_false',
                    help='ensemble only: skip timing the replicas one after another')
    ap.add_argument('--compare-steps', type=int, default=20)
    ap.add_argument('--cells-per-cutoff', type=int, default=0,
                    help='cell-list stencil width m (cells of edge >= rcut/m); 0 = library default')
    ap.add_argument('--random-flux', type=float, default=0.0, metavar='M_S',
                    help='random flux of Eq. 7 with solute mass M_S (0: off, as in the paper)')
    ap.add_argument('--lagged-av', action='store_true',
                    help='area/volume constraints from the previous step (the concurrent variant of Sec. 3.3)')
    ap.add_argument('--lanes', type=int, default=0,
                    help='lanes per particle of the pair kernel (0: timed at commit)')
    ap.add_argument('--pair-mode', type=int, default=0, choices=[0, 1, 2],
                    help='pair kernel with lists: 1 full shell, 2 half shell, 0 chosen at commit')
    ap.add_argument('--sort-mode', type=int, default=0, choices=[0, 1, 2],
                    help='list-mode sort: 1 kernel chain, 2 one thread-block cluster, 0 chosen at commit')
    ap.add_argument('--skin', type=float, default=None,
                    help='neighbour-list skin; 0 = cell mode (stencil every step); default: the library\'s')
    args = ap.parse_args()
    if args.impl == 'reference':
        return run_reference(args)
    return run_native(args)


if __name__ == '__main__':
    sys.exit(main())
