"""Seeds whose expander column 0 first draws a value that Lemire's bounded
method must reject (the branch random inputs never reach).  Built by
inverting SplitMix64's output finaliser; used by the oracle pin and by the
GPU parity test of the same branch.  Holds no arithmetic of the method."""

M64 = 1 << 64
GAMMA = 0x9e3779b97f4a7c15        # SplitMix64's state increment
COLUMN_STEP = 0xd1b54a32d192ed03  # column j's stream starts at seed + (j+1) * step
M = 6                             # rows; threshold (2^64 - 6) mod 6 = 4


def unfinalise(x):
    """Inverse of SplitMix64's output finaliser (two xor-shift-multiply
    rounds and a last xor-shift, each invertible mod 2^64)."""
    mask = M64 - 1

    def unxorshift(y, s):
        z = y
        for _ in range(64 // s + 1):
            z = y ^ (z >> s)
        return z & mask
    z = unxorshift(x, 31)
    z = (z * pow(0x94d049bb133111eb, -1, M64)) & mask
    z = unxorshift(z, 27)
    z = (z * pow(0xbf58476d1ce4e5b9, -1, M64)) & mask
    return unxorshift(z, 30)


def rejected_first_draws():
    """(x0, seed) pairs: x0 = floor(c 2^64 / 6) + 1 for c in (1, 4) leaves a
    low word x0 * 6 mod 2^64 of 2, below the threshold 4; `seed` makes it
    column 0's first draw."""
    out = []
    for c in (1, 4):
        x0 = c * M64 // M + 1
        out.append((x0, (unfinalise(x0) - GAMMA - COLUMN_STEP) % M64))
    return out
