"""Host model of the operand-stage protocol of the warp-specialised network
kernel (k_mlp_bf16_ws in csrc/gnn_bf16.cu), run on the CPU.

One producer fills tiles 0, 1, 2, ... into S stages (tile j into stage
j % S, after the stage's "empty" barrier has completed the phase of tile
j - S); NG warpgroups take tiles g, g + NG, ...; a warpgroup waits on the
stage's "full" barrier with the parity of tile j's phase, reads the tile,
and releases the stage.  An mbarrier parity wait returns once the barrier's
current phase has a parity other than the one waited for, so it tells only
the last two phases apart.

With NG <= S the parity wait alone is exact.  With NG > S a warpgroup can
ask for tile j while its stage still holds (or waits for) tile j - S, whose
phase parity is the opposite one: the plain parity wait then accepts the
wrong phase.  The kernel therefore has the producer publish the tile it
starts in each stage, and a warpgroup first waits until that word reaches
j.  The model checks both statements over random interleavings.
"""
import random

import pytest


class Barrier:
    """Phase counter with the mbarrier parity-wait rule."""

    def __init__(self):
        self.phase = 0          # number of completed phases

    def complete(self):
        self.phase += 1

    def try_wait(self, parity):
        # the phase with this parity has completed when the current
        # (incomplete) phase has the other parity
        return (self.phase & 1) != parity


def simulate(S, NG, ntiles, use_gen, seed):
    """Random interleaving of the producer and NG consumers; returns the
    list of (tile wanted, tile found) for every tile a consumer read."""
    rng = random.Random(seed)
    full = [Barrier() for _ in range(S)]
    empty = [Barrier() for _ in range(S)]
    content = [None] * S            # tile currently in each stage
    gen = [-1] * S                  # tile last started in each stage
    nxt = 0                         # producer's next tile
    state = {g: ("want", g) for g in range(NG)}   # per consumer: waiting for / holding a tile
    reads = []
    for _ in range(20000):
        actors = []
        if nxt < ntiles:
            actors.append("p")
        actors += [g for g in range(NG) if state[g][1] < ntiles]
        if not actors:
            break
        a = rng.choice(actors)
        if a == "p":
            j = nxt
            s = j % S
            if j >= S and not empty[s].try_wait(((j // S) - 1) & 1):
                continue                            # stage not yet released
            gen[s] = j
            content[s] = j                          # the copies land...
            full[s].complete()                      # ...and complete the phase
            nxt += 1
        else:
            kind, j = state[a]
            s = j % S
            if kind == "want":
                if use_gen and NG > S and gen[s] < j:
                    continue
                if not full[s].try_wait((j // S) & 1):
                    continue
                reads.append((j, content[s]))
                state[a] = ("hold", j)
            else:
                empty[s].complete()                 # the first layer has read the stage
                state[a] = ("want", j + NG)
    return reads


@pytest.mark.parametrize("S,NG", [(3, 2), (2, 2), (3, 3), (2, 3), (2, 4), (1, 3)])
def test_published_tile_word_keeps_every_read_on_its_tile(S, NG):
    for seed in range(40):
        reads = simulate(S, NG, 60, use_gen=True, seed=seed)
        assert len(reads) == 60
        assert all(want == got for want, got in reads)


@pytest.mark.parametrize("S,NG", [(3, 2), (3, 3)])
def test_parity_alone_is_exact_with_enough_stages(S, NG):
    for seed in range(40):
        reads = simulate(S, NG, 60, use_gen=False, seed=seed)
        assert all(want == got for want, got in reads)


def test_parity_alone_accepts_a_wrong_phase_with_more_warpgroups_than_stages():
    # three warpgroups over two stages (the edge update's configuration):
    # some interleaving lets a warpgroup read a tile that is not its own
    bad = 0
    for seed in range(200):
        reads = simulate(2, 3, 60, use_gen=False, seed=seed)
        bad += sum(want != got for want, got in reads)
    assert bad > 0
