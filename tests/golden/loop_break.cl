__kernel void early_exit(__global int *a, uint n)
{
    uint var0;
    uint var1;
    uint var2;
    uint var3;
    uint var4;
    uint var5;
    var0 = 0u;
    var1 = 0u;
    do {
        var2 = (var0 + 3u);
        if (var1 == n) {
            var5 = var2;
            break;
        }
        var3 = (var2 + 5u);
        var4 = (var1 + 1u);
        var5 = var3;
        var0 = var3;
        var1 = var4;
    } while (var4 < 4u);
    a[get_local_id(0)] = (int)var5;
}
